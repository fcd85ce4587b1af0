// Decoder backward (Sec. 3.2, Eq. offsets and Eq. mlp): shapes, argument block, scratch
// layout and the per-Gaussian output gradient shared by the FP32 and the tensor-core row
// passes (grad.cu, decode_bwd_tc.cu).
#pragma once

#include "internal.cuh"

namespace ogs {
namespace db {

constexpr int kDbThreads = 128;
constexpr int kF = 32;
constexpr int kH = 32;
constexpr int kDin = kF + 4;
constexpr int kK = 10;
constexpr int kNW1 = 3 * kH * kDin;                       // 3456
constexpr int kNB1 = 3 * kH;                              // 96
constexpr int kNOut = 11 * kK;                            // 110 (10 + 30 + 70)
constexpr int kNW2 = kNOut * kH;                          // 3520
constexpr int kNWeights = kNW1 + kNB1 + kNW2 + kNOut;     // 7182

// offsets of the decoder gradients inside one flat partial row:
//   dw1 [3][H][Din] | db1 [3][H] | dw2_op [k][H] | dw2_col [3k][H] | dw2_cov [7k][H] |
//   db2_op [k] | db2_col [3k] | db2_cov [7k]
constexpr int kOffB1 = kNW1;
constexpr int kOffW2 = kOffB1 + kNB1;
constexpr int kOffB2 = kOffW2 + kNW2;

// per-anchor rows handed from the row pass to the weight pass (f32, 16-byte aligned rows)
constexpr int kRowY = 112;    // dL/dy of the 110 stacked outputs (+2 zero)
constexpr int kRowH = 96;     // hidden activations of the three decoders
constexpr int kRowP = 96;     // dL/d(pre-activation) of the three decoders
constexpr int kRowZ = 40;     // decoder input z (36, +4 zero)

struct DbArgs {
    const float* pos;
    const float* feat;
    const float* offs;
    const float* lv;
    const uint32_t* sel_idx;
    const float* sel_w;
    const ogs_counts* counts;
    ogs_mlp mlp;
    Cam cam;
    const float* dmeans;
    const float* dscales;
    const float* dquats;
    const float* drec;
    float* dfeat;
    float* doffs;
    float* dlv;
    float* rowY;         // [sel_cap][kRowY]
    float* rowH;         // [sel_cap][kRowH]
    float* rowP;         // [sel_cap][kRowP]
    float* rowZ;         // [sel_cap][kRowZ]
    float* partial;      // [kDbBlocks][kNWeights]
    float* dapp;         // f32[N][A] appearance code gradients (+=), with codes only
};

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + __expf(-x)); }

// out rows of decoder m (opacity 0, colour 1, covariance 2) inside the 110 stacked outputs
__device__ __forceinline__ int out_base(int m) { return m == 0 ? 0 : (m == 1 ? kK : 4 * kK); }
__device__ __forceinline__ int dec_of(int row) { return row < kK ? 0 : (row < 4 * kK ? 1 : 2); }

// Gradient of the loss w.r.t. the outputs y of decoder m for Gaussian i of anchor j (row
// g = r k + i of the Gaussian arrays): opacity w tanh (zero where the opacity was dropped),
// colour sigmoid, scale l_v sigmoid, unit quaternion; the scale and position terms of l_v and
// the offsets are accumulated here (dlv, doffs).
__device__ __forceinline__ void gaussian_dy(const DbArgs& a, int m, size_t g, uint32_t j, int i,
                                            float w, const float (&lvv)[3], const float* y,
                                            float* dy, float (&dlv)[3]) {
    if (m == 0) {
        const float th = tanhf(y[0]);
        dy[0] = w * th > 0.f ? a.drec[9 * g + 5] * w * (1.f - th * th) : 0.f;
    } else if (m == 1) {
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const float sg = sigm(y[e]);
            dy[e] = a.drec[9 * g + 6 + e] * sg * (1.f - sg);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const float sg = sigm(y[e]);
            const float gsc = a.dscales[3 * g + e];
            dlv[e] += gsc * sg;
            dy[e] = gsc * lvv[e] * sg * (1.f - sg);
        }
        const float n2 = y[3] * y[3] + y[4] * y[4] + y[5] * y[5] + y[6] * y[6];
        const float inv = 1.0f / sqrtf(n2);
        const float4 gq = *reinterpret_cast<const float4*>(a.dquats + 4 * g);
        const float qn[4] = {y[3] * inv, y[4] * inv, y[5] * inv, y[6] * inv};
        const float gqa[4] = {gq.x, gq.y, gq.z, gq.w};
        const float dot = qn[0] * gqa[0] + qn[1] * gqa[1] + qn[2] * gqa[2] + qn[3] * gqa[3];
#pragma unroll
        for (int e = 0; e < 4; ++e) dy[3 + e] = (gqa[e] - qn[e] * dot) * inv;
        // positions: mu = x_v + O * l_v
        const float* O = a.offs + ((size_t)j * kK + i) * 3;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const float gmu = a.dmeans[3 * g + e];
            a.doffs[((size_t)j * kK + i) * 3 + e] += gmu * lvv[e];
            dlv[e] += gmu * O[e];
        }
    }
}

constexpr int kDbBlocks = 2 * kSmCount;

// partial sums of the appearance weight gradients: one kH x kMaxApp row per block
constexpr int kAppItems = kH * kMaxApp;

struct DbScratch {
    float* partial;
    float *rowY, *rowH, *rowP, *rowZ;
    float* partial_app;  // [kDbBlocks][kAppItems]
};

inline size_t db_layout(int64_t sel_cap, void* base, DbScratch* s) {
    Carver cv(base);
    DbScratch t;
    const size_t n = (size_t)(sel_cap > 0 ? sel_cap : 1);
    t.partial = cv.take<float>((size_t)kDbBlocks * kNWeights);
    t.rowY = cv.take<float>(n * kRowY);
    t.rowH = cv.take<float>(n * kRowH);
    t.rowP = cv.take<float>(n * kRowP);
    t.rowZ = cv.take<float>(n * kRowZ);
    t.partial_app = cv.take<float>((size_t)kDbBlocks * kAppItems);
    if (s) *s = t;
    return cv.off + 256;
}

// Weight pass + fixed-order reduction over the rows written by a row pass (grad.cu); with
// appearance codes (a.mlp.A > 0) also the code weights' gradient dmlp.w1_app.
cudaError_t launch_weight_pass(const DbArgs& a, const DbScratch& s, const ogs_mlp& dmlp,
                               cudaStream_t st);

}  // namespace db
}  // namespace ogs
