// Backward of the EWA projection (Sec. 3.1, Eq. 1) and of the neural-Gaussian decoders
// (Sec. 3.2, Eq. offsets and Eq. mlp), plus the L1 photometric loss and a fused Adam update.
//
// project_bwd: one thread per Gaussian; recomputes the forward quantities and chains
//   d(u, v, conic) -> d(mean, scale, unit quaternion).
// decode_bwd: one thread per selected anchor recomputes its three decoders and produces
//   d(feature), d(offsets), d(l_v); the weight gradients are block-level products
//   dY^T H and dPre^T Z of the block's anchors (staged in shared memory), each element owned
//   by one thread, written as per-block partials and summed by a deterministic reduction.
#include "internal.cuh"

namespace ogs {
namespace {

constexpr int kPbThreads = 256;

struct PbArgs {
    ogs_gaussians g;
    const uint32_t* count;
    int64_t n_fixed;
    int rel;
    Cam cam;
    const uint2* rect;
    const float* drec;     // [G][9]: du dv da db dc do dr dg db
    float* dmeans;         // [G][3]
    float* dscales;        // [G][3]
    float* dquats;         // [G][4]
};

__global__ void __launch_bounds__(kPbThreads) project_bwd_kernel(PbArgs a) {
    const Cam& c = a.cam;
    const int64_t n = a.count ? (int64_t)*a.count : a.n_fixed;
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < n;
         gi += (int64_t)gridDim.x * blockDim.x) {
        float gm0 = 0.f, gm1 = 0.f, gm2 = 0.f, gs0 = 0.f, gs1 = 0.f, gs2 = 0.f;
        float gq0 = 0.f, gq1 = 0.f, gq2 = 0.f, gq3 = 0.f;
        const uint2 rc = a.rect[gi];
        const bool vis = (rc.x & 0xFFFFu) < (rc.y & 0xFFFFu);
        if (vis) {
            const float* dr = a.drec + 9 * gi;
            const float du = dr[0], dv = dr[1], dca = dr[2], dcb = dr[3], dcc = dr[4];
            float m0 = a.g.means[3 * gi], m1 = a.g.means[3 * gi + 1], m2 = a.g.means[3 * gi + 2];
            if (!a.rel) { m0 -= c.c[0]; m1 -= c.c[1]; m2 -= c.c[2]; }
            const float px = c.R[0] * m0 + c.R[1] * m1 + c.R[2] * m2;
            const float py = c.R[3] * m0 + c.R[4] * m1 + c.R[5] * m2;
            const float pz = c.R[6] * m0 + c.R[7] * m1 + c.R[8] * m2;
            const float4 q = *reinterpret_cast<const float4*>(a.g.quats + 4 * gi);
            const float s[3] = {a.g.scales[3 * gi], a.g.scales[3 * gi + 1], a.g.scales[3 * gi + 2]};
            const float w = q.x, x = q.y, y = q.z, z = q.w;
            const float Rq[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                                 2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                                 2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
            float M[9], S[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k) M[3 * r + k] = Rq[3 * r + k] * s[k];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    S[3 * r + k] = M[3 * r] * M[3 * k] + M[3 * r + 1] * M[3 * k + 1] + M[3 * r + 2] * M[3 * k + 2];
            const float iz = 1.0f / pz;
            const float xz = px * iz, yz = py * iz;
            const bool clx = xz < -c.limx || xz > c.limx, cly = yz < -c.limy || yz > c.limy;
            const float tx = fminf(fmaxf(xz, -c.limx), c.limx) * pz;
            const float ty = fminf(fmaxf(yz, -c.limy), c.limy) * pz;
            const float J[6] = {c.fx * iz, 0.f, -c.fx * tx * iz * iz, 0.f, c.fy * iz, -c.fy * ty * iz * iz};
            float T[6];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    T[3 * r + k] = J[3 * r] * c.R[k] + J[3 * r + 1] * c.R[3 + k] + J[3 * r + 2] * c.R[6 + k];
            float TS[6];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    TS[3 * r + k] = T[3 * r] * S[k] + T[3 * r + 1] * S[3 + k] + T[3 * r + 2] * S[6 + k];
            const float A = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + 0.3f;
            const float B = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
            const float Cc = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + 0.3f;
            const float id = 1.0f / (A * Cc - B * B);
            const float ka = Cc * id, kb = -B * id, kc = A * id;
            // dL/dM (M = cov2 + 0.3 I) = -K G K with G the symmetric gradient of the conic
            const float g00 = dca, g01 = 0.5f * dcb, g11 = dcc;
            const float t00 = ka * g00 + kb * g01, t01 = ka * g01 + kb * g11;
            const float t10 = kb * g00 + kc * g01, t11 = kb * g01 + kc * g11;
            const float G00 = -(t00 * ka + t01 * kb), G01 = -(t00 * kb + t01 * kc);
            const float G11 = -(t10 * kb + t11 * kc);
            const float Gm[4] = {G00, G01, G01, G11};
            // dL/dSigma = T^T Gm T ; dL/dT = 2 Gm T Sigma
            float gS[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    gS[3 * r + k] = T[r] * (Gm[0] * T[k] + Gm[1] * T[3 + k]) +
                                    T[3 + r] * (Gm[2] * T[k] + Gm[3] * T[3 + k]);
            float gT[6];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    gT[3 * r + k] = 2.f * (Gm[2 * r] * TS[k] + Gm[2 * r + 1] * TS[3 + k]);
            float gJ[6];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    gJ[3 * r + k] = gT[3 * r] * c.R[3 * k] + gT[3 * r + 1] * c.R[3 * k + 1] +
                                    gT[3 * r + 2] * c.R[3 * k + 2];
            const float iz2 = iz * iz, iz3 = iz2 * iz;
            float gp0 = 0.f, gp1 = 0.f, gp2 = 0.f;
            gp2 += gJ[0] * (-c.fx * iz2) + gJ[4] * (-c.fy * iz2);
            if (!clx) { gp0 += gJ[2] * (-c.fx * iz2); gp2 += gJ[2] * (2.f * c.fx * px * iz3); }
            else gp2 += gJ[2] * (c.fx * (xz < 0.f ? -c.limx : c.limx) * iz2);
            if (!cly) { gp1 += gJ[5] * (-c.fy * iz2); gp2 += gJ[5] * (2.f * c.fy * py * iz3); }
            else gp2 += gJ[5] * (c.fy * (yz < 0.f ? -c.limy : c.limy) * iz2);
            gp0 += du * c.fx * iz;
            gp2 += du * (-c.fx * px * iz2);
            gp1 += dv * c.fy * iz;
            gp2 += dv * (-c.fy * py * iz2);
            gm0 = c.R[0] * gp0 + c.R[3] * gp1 + c.R[6] * gp2;
            gm1 = c.R[1] * gp0 + c.R[4] * gp1 + c.R[7] * gp2;
            gm2 = c.R[2] * gp0 + c.R[5] * gp1 + c.R[8] * gp2;
            // Sigma = M M^T, M = R(q) S:  dL/dM = 2 gS M
            float gR[9];
            float gsv[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float gM = 2.f * (gS[3 * r] * M[k] + gS[3 * r + 1] * M[3 + k] + gS[3 * r + 2] * M[6 + k]);
                    gsv[k] += gM * Rq[3 * r + k];
                    gR[3 * r + k] = gM * s[k];
                }
            gs0 = gsv[0]; gs1 = gsv[1]; gs2 = gsv[2];
            gq0 = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
            gq1 = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] +
                         w * gR[7] - 2.f * x * gR[8]);
            gq2 = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] +
                         z * gR[7] - 2.f * y * gR[8]);
            gq3 = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] +
                         y * gR[5] + x * gR[6] + y * gR[7]);
        }
        a.dmeans[3 * gi] = gm0; a.dmeans[3 * gi + 1] = gm1; a.dmeans[3 * gi + 2] = gm2;
        a.dscales[3 * gi] = gs0; a.dscales[3 * gi + 1] = gs1; a.dscales[3 * gi + 2] = gs2;
        *reinterpret_cast<float4*>(a.dquats + 4 * gi) = make_float4(gq0, gq1, gq2, gq3);
    }
}

// ---------------------------------------------------------------------------------------
// decoder backward
// ---------------------------------------------------------------------------------------

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
    float* partial;      // [gridDim.x][kNWeights]
};

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + __expf(-x)); }

// out rows of decoder m (opacity 0, colour 1, covariance 2) inside the 110 stacked outputs
__device__ __forceinline__ int out_base(int m) { return m == 0 ? 0 : (m == 1 ? kK : 4 * kK); }
__device__ __forceinline__ int out_count(int m) { return m == 0 ? kK : (m == 1 ? 3 * kK : 7 * kK); }

__global__ void __launch_bounds__(kDbThreads) decode_bwd_kernel(DbArgs a) {
    extern __shared__ __align__(16) float sm[];
    float* acc = sm;                                   // [kNWeights] block accumulators
    float* sZ = acc + kNWeights;                       // [threads][kDin]
    float* sH = sZ + kDbThreads * kDin;                // [threads][kH]
    float* sP = sH + kDbThreads * kH;                  // [threads][kH]  d pre-activation
    float* sY = sP + kDbThreads * kH;                  // [threads][7k]  d outputs of one decoder
    for (int i = threadIdx.x; i < kNWeights; i += blockDim.x) acc[i] = 0.f;
    const uint32_t M = a.counts->n_selected;
    const Cam& c = a.cam;
    const int t = threadIdx.x;
    const float* W1 = a.mlp.w1;
    for (uint32_t base = blockIdx.x * kDbThreads; base < M; base += gridDim.x * kDbThreads) {
        const uint32_t r = base + t;
        const bool valid = r < M;
        uint32_t j = 0;
        float w = 0.f, z[kDin], dz[kF], lvv[3] = {0.f, 0.f, 0.f}, dlv[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < kF; ++i) dz[i] = 0.f;
        if (valid) {
            j = a.sel_idx[r];
            w = a.sel_w[r];
#pragma unroll
            for (int i = 0; i < kF; ++i) z[i] = a.feat[(size_t)j * kF + i];
            float dv[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                dv[q] = a.pos[3 * (size_t)j + q] - c.c[q];
                lvv[q] = a.lv[3 * (size_t)j + q];
            }
            const float d = sqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
            z[kF] = dv[0] / d; z[kF + 1] = dv[1] / d; z[kF + 2] = dv[2] / d; z[kF + 3] = d;
        } else {
#pragma unroll
            for (int i = 0; i < kDin; ++i) z[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < kDin; ++i) sZ[t * kDin + i] = z[i];
        const size_t g0 = (size_t)r * kK;
        for (int m = 0; m < 3; ++m) {
            const float* w1 = W1 + m * kH * kDin;
            const float* b1 = a.mlp.b1 + m * kH;
            float h[kH], dh[kH];
            unsigned mask = 0;
#pragma unroll
            for (int o = 0; o < kH; ++o) {
                float p = b1[o];
#pragma unroll
                for (int i = 0; i < kDin; ++i) p = fmaf(w1[o * kDin + i], z[i], p);
                h[o] = fmaxf(p, 0.f);
                mask |= (p > 0.f ? 1u : 0u) << o;
                dh[o] = 0.f;
            }
            const int nout = out_count(m);
            const float* w2 = m == 0 ? a.mlp.w2_op : (m == 1 ? a.mlp.w2_col : a.mlp.w2_cov);
            const float* b2 = m == 0 ? a.mlp.b2_op : (m == 1 ? a.mlp.b2_col : a.mlp.b2_cov);
            // per Gaussian: outputs, their gradients, and the chain into the hidden layer
            for (int i = 0; i < kK; ++i) {
                const int per = m == 0 ? 1 : (m == 1 ? 3 : 7);
                float y[7], dy[7];
#pragma unroll
                for (int e = 0; e < 7; ++e) {
                    if (e >= per) { y[e] = 0.f; continue; }
                    const int row = per * i + e;
                    float v = b2[row];
#pragma unroll
                    for (int o = 0; o < kH; ++o) v = fmaf(w2[row * kH + o], h[o], v);
                    y[e] = v;
                }
#pragma unroll
                for (int e = 0; e < 7; ++e) dy[e] = 0.f;
                if (valid) {
                    const size_t g = g0 + i;
                    if (m == 0) {
                        const float th = tanhf(y[0]);
                        if (w * th > 0.f) dy[0] = a.drec[9 * g + 5] * w * (1.f - th * th);
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
#pragma unroll
                for (int e = 0; e < 7; ++e) {
                    if (e >= per) continue;
                    const int row = per * i + e;
                    sY[t * (7 * kK) + row] = dy[e];
#pragma unroll
                    for (int o = 0; o < kH; ++o) dh[o] = fmaf(w2[row * kH + o], dy[e], dh[o]);
                }
            }
            // hidden: relu mask, then into the input features
#pragma unroll
            for (int o = 0; o < kH; ++o) {
                const float dp = (mask >> o) & 1u ? dh[o] : 0.f;
                sH[t * kH + o] = h[o];
                sP[t * kH + o] = dp;
#pragma unroll
                for (int i = 0; i < kF; ++i) dz[i] = fmaf(w1[o * kDin + i], dp, dz[i]);
            }
            __syncthreads();
            // block products: dW2_m += dY^T H, db2_m += sum dY, dW1_m += dP^T Z, db1_m += sum dP
            const int nv = min((uint32_t)kDbThreads, M - base);
            float* aw2 = acc + kOffW2 + out_base(m) * kH;
            float* ab2 = acc + kOffB2 + out_base(m);
            for (int e = t; e < nout * kH; e += kDbThreads) {
                const int row = e / kH, o = e % kH;
                float s = 0.f;
                for (int q = 0; q < nv; ++q) s = fmaf(sY[q * (7 * kK) + row], sH[q * kH + o], s);
                aw2[e] += s;
            }
            for (int e = t; e < nout; e += kDbThreads) {
                float s = 0.f;
                for (int q = 0; q < nv; ++q) s += sY[q * (7 * kK) + e];
                ab2[e] += s;
            }
            float* aw1 = acc + m * kH * kDin;
            float* ab1 = acc + kOffB1 + m * kH;
            for (int e = t; e < kH * kDin; e += kDbThreads) {
                const int o = e / kDin, i = e % kDin;
                float s = 0.f;
                for (int q = 0; q < nv; ++q) s = fmaf(sP[q * kH + o], sZ[q * kDin + i], s);
                aw1[e] += s;
            }
            for (int e = t; e < kH; e += kDbThreads) {
                float s = 0.f;
                for (int q = 0; q < nv; ++q) s += sP[q * kH + e];
                ab1[e] += s;
            }
            __syncthreads();
        }
        if (valid) {
#pragma unroll
            for (int i = 0; i < kF; ++i) a.dfeat[(size_t)j * kF + i] += dz[i];
#pragma unroll
            for (int e = 0; e < 3; ++e) a.dlv[3 * (size_t)j + e] += dlv[e];
        }
    }
    __syncthreads();
    float* out = a.partial + (size_t)blockIdx.x * kNWeights;
    for (int i = threadIdx.x; i < kNWeights; i += blockDim.x) out[i] = acc[i];
}

// dmlp[e] += sum over blocks of partial[b][e] (fixed order: deterministic)
__global__ void reduce_partials(const float* __restrict__ partial, int nblocks, ogs_mlp grads) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kNWeights; e += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * kNWeights + e];
        float* dst;
        int i = e;
        if (i < kNW1) dst = const_cast<float*>(grads.w1) + i;
        else if ((i -= kNW1) < kNB1) dst = const_cast<float*>(grads.b1) + i;
        else if ((i -= kNB1) < kK * kH) dst = const_cast<float*>(grads.w2_op) + i;
        else if ((i -= kK * kH) < 3 * kK * kH) dst = const_cast<float*>(grads.w2_col) + i;
        else if ((i -= 3 * kK * kH) < 7 * kK * kH) dst = const_cast<float*>(grads.w2_cov) + i;
        else if ((i -= 7 * kK * kH) < kK) dst = const_cast<float*>(grads.b2_op) + i;
        else if ((i -= kK) < 3 * kK) dst = const_cast<float*>(grads.b2_col) + i;
        else dst = const_cast<float*>(grads.b2_cov) + (i - 3 * kK);
        *dst += s;
    }
}

constexpr int kDbBlocks = 2 * kSmCount;

size_t decode_bwd_smem() {
    return sizeof(float) * (kNWeights + kDbThreads * (kDin + kH + kH + 7 * kK));
}

// ---------------------------------------------------------------------------------------
// loss and optimiser
// ---------------------------------------------------------------------------------------

// L = mean |img - target|; dimg = sign(img - target) / n; loss accumulated into *loss
__global__ void l1_kernel(const float* __restrict__ img, const float* __restrict__ target,
                          int64_t n, float scale, float* __restrict__ dimg,
                          float* __restrict__ loss) {
    float s = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float d = img[i] - target[i];
        s += fabsf(d);
        dimg[i] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane_id() == 0 && loss) atomicAdd(loss, s * scale);
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2, int zero_grad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        if (zero_grad) grad[i] = 0.f;
    }
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" ogs_status ogs_project_bwd(const ogs_gaussians* g, int64_t n_gauss, int32_t means_relative,
                                      const ogs_camera* cam, const uint32_t* rect, const float* drec,
                                      float* dmeans, float* dscales, float* dquats,
                                      const ogs_counts* counts, void* stream) {
    if (!g || !cam || !rect || !drec || !dmeans || !dscales || !dquats || n_gauss < 0)
        return OGS_ERR_ARG;
    if (!aligned(g->quats, 16) || !aligned(dquats, 16) || !aligned(rect, 8)) return OGS_ERR_ARG;
    if (n_gauss == 0) return OGS_OK;
    PbArgs a{*g, counts ? &counts->n_gaussians : nullptr, n_gauss, means_relative, make_cam(*cam),
             reinterpret_cast<const uint2*>(rect), drec, dmeans, dscales, dquats};
    project_bwd_kernel<<<stride_grid(n_gauss, kPbThreads, 8), kPbThreads, 0,
                         (cudaStream_t)stream>>>(a);
    return launch_status();
}

extern "C" size_t ogs_decode_bwd_scratch_bytes(void) {
    return sizeof(float) * (size_t)kDbBlocks * kNWeights + 256;
}

extern "C" ogs_status ogs_decode_bwd(const float* pos, const float* feat, const float* offs,
                                     const float* lv, int64_t N, const ogs_mlp* mlp,
                                     const ogs_camera* cam, const uint32_t* sel_idx,
                                     const float* sel_w, const ogs_counts* counts,
                                     const float* dmeans, const float* dscales,
                                     const float* dquats, const float* drec, float* dfeat,
                                     float* doffs, float* dlv, const ogs_mlp* dmlp, void* scratch,
                                     size_t scratch_bytes, void* stream) {
    if (!pos || !feat || !offs || !lv || !mlp || !cam || !sel_idx || !sel_w || !counts ||
        !dmeans || !dscales || !dquats || !drec || !dfeat || !doffs || !dlv || !dmlp || !scratch)
        return OGS_ERR_ARG;
    if (mlp->F != kF || mlp->H != kH || mlp->k != kK || N < 0) return OGS_ERR_ARG;
    if (!dmlp->w1 || !dmlp->b1 || !dmlp->w2_op || !dmlp->b2_op || !dmlp->w2_col ||
        !dmlp->b2_col || !dmlp->w2_cov || !dmlp->b2_cov)
        return OGS_ERR_ARG;
    if (scratch_bytes < ogs_decode_bwd_scratch_bytes() || !aligned(scratch, 16) ||
        !aligned(dquats, 16))
        return OGS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    size_t smem = decode_bwd_smem();
    if (cudaFuncSetAttribute(decode_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return OGS_ERR_CUDA;
    DbArgs a{pos, feat, offs, lv, sel_idx, sel_w, counts, *mlp, make_cam(*cam), dmeans, dscales,
             dquats, drec, dfeat, doffs, dlv, (float*)scratch};
    decode_bwd_kernel<<<kDbBlocks, kDbThreads, smem, st>>>(a);
    reduce_partials<<<(kNWeights + 255) / 256, 256, 0, st>>>((const float*)scratch, kDbBlocks, *dmlp);
    return launch_status();
}

extern "C" ogs_status ogs_loss_l1(const float* img, const float* target, int64_t n, float* dimg,
                                  float* loss, void* stream) {
    if (!img || !target || !dimg || n <= 0) return OGS_ERR_ARG;
    l1_kernel<<<stride_grid(n, 256, 8), 256, 0, (cudaStream_t)stream>>>(img, target, n,
                                                                         1.0f / (float)n, dimg, loss);
    return launch_status();
}

extern "C" ogs_status ogs_adam(float* param, float* grad, float* m, float* v, int64_t n, float lr,
                               float beta1, float beta2, float eps, int32_t step,
                               int32_t zero_grad, void* stream) {
    if (!param || !grad || !m || !v || n < 0 || step < 1) return OGS_ERR_ARG;
    if (n == 0) return OGS_OK;
    const float bc1 = 1.f - powf(beta1, (float)step), bc2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<stride_grid(n, 256, 8), 256, 0, (cudaStream_t)stream>>>(
        param, grad, m, v, n, lr, beta1, beta2, eps, bc1, bc2, zero_grad);
    return launch_status();
}
