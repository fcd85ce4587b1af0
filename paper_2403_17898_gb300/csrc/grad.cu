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
#include "decode_bwd.cuh"
#include "tc.cuh"

namespace ogs {
namespace {

using namespace db;

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

// Row pass: two threads per selected anchor recompute its decoders (weights in shared memory,
// broadcast reads) and chain the per-Gaussian gradients into dy (110), the hidden
// pre-activation gradients dp (96) and the feature gradient (dfeat, doffs, dlv accumulate;
// each anchor appears once per view, so no atomics).  The CTA's first two warps take the
// opacity and colour decoders of 64 anchors, the last two the covariance decoder (and the
// position terms) of the same anchors: equal work, no divergence inside a warp; the two
// feature-gradient halves meet in shared memory.  dy, h, dp and z are written as rows for
// the weight pass.  Layer 1 runs in outer-product form over a streamed input (only the 32
// hidden accumulators live in registers), so a thread keeps h, dh and dz (96 values).
constexpr int kRowAnchors = kDbThreads / 2;

template <bool APP>
__global__ void __launch_bounds__(kDbThreads, 3) decode_bwd_rows(DbArgs a) {
    __shared__ __align__(16) float sW1t[3 * kDin * kH];   // [m][i][o]
    __shared__ __align__(16) float sW1[3 * kH * kDin];    // [m][o][i]
    __shared__ float sB1[kNB1];
    __shared__ __align__(16) float sW2[kNOut * kH];
    __shared__ float sB2[kNOut];
    __shared__ float sDz[kRowAnchors][kF + 1];
    __shared__ __align__(16) float sWa[kH * kMaxApp];     // appearance weights [o][c], padded
    const int napp = a.mlp.A;
    for (int e = threadIdx.x; e < kH * kMaxApp; e += kDbThreads) {
        const int o = e / kMaxApp, q = e % kMaxApp;
        sWa[e] = q < napp ? a.mlp.w1_app[o * napp + q] : 0.f;
    }
    for (int e = threadIdx.x; e < 3 * kH * kDin; e += kDbThreads) {
        const float v = a.mlp.w1[e];
        sW1[e] = v;
        const int m = e / (kH * kDin), o = (e / kDin) % kH, i = e % kDin;
        sW1t[(m * kDin + i) * kH + o] = v;
    }
    for (int e = threadIdx.x; e < kNOut * kH; e += kDbThreads)
        sW2[e] = e < kK * kH ? a.mlp.w2_op[e]
                             : (e < 4 * kK * kH ? a.mlp.w2_col[e - kK * kH]
                                                : a.mlp.w2_cov[e - 4 * kK * kH]);
    for (int e = threadIdx.x; e < kNB1; e += kDbThreads) sB1[e] = a.mlp.b1[e];
    for (int e = threadIdx.x; e < kNOut; e += kDbThreads)
        sB2[e] = e < kK ? a.mlp.b2_op[e] : (e < 4 * kK ? a.mlp.b2_col[e - kK] : a.mlp.b2_cov[e - 4 * kK]);
    __syncthreads();
    const uint32_t M = a.counts->n_selected;
    const Cam& c = a.cam;
    const bool cov_half = threadIdx.x >= kRowAnchors;        // warp-uniform
    const int slot = threadIdx.x - (cov_half ? kRowAnchors : 0);
    const int m_lo = cov_half ? 2 : 0, m_hi = cov_half ? 3 : 2;
    for (uint32_t base = blockIdx.x * kRowAnchors; base < M; base += gridDim.x * kRowAnchors) {
        const uint32_t r = base + slot;
        const bool valid = r < M;
        float dz[kF];
#pragma unroll
        for (int i = 0; i < kF; ++i) dz[i] = 0.f;
        if (valid) {
        const uint32_t j = a.sel_idx[r];
        const float w = a.sel_w[r];
        const float4* f4 = reinterpret_cast<const float4*>(a.feat + (size_t)j * kF);
        float lvv[3], dlv[3] = {0.f, 0.f, 0.f}, zc[4];
        float dv[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            dv[q] = a.pos[3 * (size_t)j + q] - c.c[q];
            lvv[q] = a.lv[3 * (size_t)j + q];
        }
        const float d = sqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        zc[0] = dv[0] / d; zc[1] = dv[1] / d; zc[2] = dv[2] / d; zc[3] = d;
        if (!cov_half) {
            float4* zr = reinterpret_cast<float4*>(a.rowZ + (size_t)r * kRowZ);
#pragma unroll
            for (int i = 0; i < kF / 4; ++i) zr[i] = f4[i];
            zr[kF / 4] = make_float4(zc[0], zc[1], zc[2], zc[3]);
            zr[kF / 4 + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float* yrow = a.rowY + (size_t)r * kRowY;
        if (cov_half) {
            yrow[kNOut] = 0.f;
            yrow[kNOut + 1] = 0.f;
        }
        const size_t g0 = (size_t)r * kK;
#pragma unroll 1
        for (int m = m_lo; m < m_hi; ++m) {
            float h[kH], dh[kH];
#pragma unroll
            for (int o = 0; o < kH; ++o) h[o] = sB1[m * kH + o];
            // layer 1, outer-product form: h += W1[:, i] z_i over the streamed input
#pragma unroll 1
            for (int i4 = 0; i4 < kDin / 4; ++i4) {
                const float4 zv = i4 < kF / 4 ? f4[i4] : make_float4(zc[0], zc[1], zc[2], zc[3]);
                const float zz[4] = {zv.x, zv.y, zv.z, zv.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float4* col = reinterpret_cast<const float4*>(sW1t + (m * kDin + 4 * i4 + u) * kH);
#pragma unroll
                    for (int q = 0; q < kH / 4; ++q) {
                        const float4 wv = col[q];
                        h[4 * q] = fmaf(wv.x, zz[u], h[4 * q]);
                        h[4 * q + 1] = fmaf(wv.y, zz[u], h[4 * q + 1]);
                        h[4 * q + 2] = fmaf(wv.z, zz[u], h[4 * q + 2]);
                        h[4 * q + 3] = fmaf(wv.w, zz[u], h[4 * q + 3]);
                    }
                }
            }
            if (APP && m == 1) {           // the colour decoder also sees the code (Sec. 4.4)
                float code[kMaxApp];
#pragma unroll
                for (int q = 0; q < kMaxApp; ++q)
                    code[q] = q < napp ? a.mlp.app[(size_t)j * napp + q] : 0.f;
#pragma unroll
                for (int o = 0; o < kH; ++o) {
                    float v = h[o];
#pragma unroll
                    for (int q = 0; q < kMaxApp; ++q) v = fmaf(sWa[o * kMaxApp + q], code[q], v);
                    h[o] = v;
                }
            }
            uint32_t mask = 0;
#pragma unroll
            for (int o = 0; o < kH; ++o) {
                mask |= (h[o] > 0.f ? 1u : 0u) << o;
                h[o] = fmaxf(h[o], 0.f);
                dh[o] = 0.f;
            }
            {
                float4* hr = reinterpret_cast<float4*>(a.rowH + (size_t)r * kRowH + m * kH);
#pragma unroll
                for (int i = 0; i < kH / 4; ++i)
                    hr[i] = make_float4(h[4 * i], h[4 * i + 1], h[4 * i + 2], h[4 * i + 3]);
            }
            const int per = m == 0 ? 1 : (m == 1 ? 3 : 7);
#pragma unroll 1
            for (int i = 0; i < kK; ++i) {
                float y[7], dy[7];
#pragma unroll
                for (int e = 0; e < 7; ++e) {
                    y[e] = 0.f;
                    dy[e] = 0.f;
                    if (e < per) {
                        const int row = out_base(m) + per * i + e;
                        const float4* wr = reinterpret_cast<const float4*>(sW2 + row * kH);
                        float v = sB2[row];
#pragma unroll
                        for (int q = 0; q < kH / 4; ++q) {
                            const float4 wv = wr[q];
                            v = fmaf(wv.x, h[4 * q], v);
                            v = fmaf(wv.y, h[4 * q + 1], v);
                            v = fmaf(wv.z, h[4 * q + 2], v);
                            v = fmaf(wv.w, h[4 * q + 3], v);
                        }
                        y[e] = v;
                    }
                }
                gaussian_dy(a, m, g0 + i, j, i, w, lvv, y, dy, dlv);
#pragma unroll
                for (int e = 0; e < 7; ++e) {
                    if (e < per) {
                        const int row = out_base(m) + per * i + e;
                        yrow[row] = dy[e];
                        const float4* wr = reinterpret_cast<const float4*>(sW2 + row * kH);
#pragma unroll
                        for (int q = 0; q < kH / 4; ++q) {
                            const float4 wv = wr[q];
                            dh[4 * q] = fmaf(wv.x, dy[e], dh[4 * q]);
                            dh[4 * q + 1] = fmaf(wv.y, dy[e], dh[4 * q + 1]);
                            dh[4 * q + 2] = fmaf(wv.z, dy[e], dh[4 * q + 2]);
                            dh[4 * q + 3] = fmaf(wv.w, dy[e], dh[4 * q + 3]);
                        }
                    }
                }
            }
            // through the ReLU, then into the features: dz_i += sum_o W1[o][i] dp_o
#pragma unroll
            for (int o = 0; o < kH; ++o) dh[o] = (mask >> o) & 1u ? dh[o] : 0.f;
            {
                float4* pr = reinterpret_cast<float4*>(a.rowP + (size_t)r * kRowP + m * kH);
#pragma unroll
                for (int i = 0; i < kH / 4; ++i)
                    pr[i] = make_float4(dh[4 * i], dh[4 * i + 1], dh[4 * i + 2], dh[4 * i + 3]);
            }
            if (APP && m == 1) {           // code gradient: dapp_c += sum_o Wa[o][c] dp_o
#pragma unroll
                for (int q = 0; q < kMaxApp; ++q) {
                    if (q < napp) {
                        float v = 0.f;
#pragma unroll
                        for (int o = 0; o < kH; ++o) v = fmaf(sWa[o * kMaxApp + q], dh[o], v);
                        a.dapp[(size_t)j * napp + q] += v;
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < kH; ++o) {
                const float4* wr = reinterpret_cast<const float4*>(sW1 + (m * kH + o) * kDin);
#pragma unroll
                for (int i = 0; i < kF / 4; ++i) {
                    const float4 wv = wr[i];
                    dz[4 * i] = fmaf(wv.x, dh[o], dz[4 * i]);
                    dz[4 * i + 1] = fmaf(wv.y, dh[o], dz[4 * i + 1]);
                    dz[4 * i + 2] = fmaf(wv.z, dh[o], dz[4 * i + 2]);
                    dz[4 * i + 3] = fmaf(wv.w, dh[o], dz[4 * i + 3]);
                }
            }
        }
        if (cov_half) {
#pragma unroll
            for (int i = 0; i < kF; ++i) sDz[slot][i] = dz[i];
#pragma unroll
            for (int e = 0; e < 3; ++e) a.dlv[3 * (size_t)j + e] += dlv[e];
        }
        }
        __syncthreads();
        if (valid && !cov_half) {
            const uint32_t j = a.sel_idx[r];
            float4* df = reinterpret_cast<float4*>(a.dfeat + (size_t)j * kF);
#pragma unroll
            for (int i = 0; i < kF / 4; ++i) {
                float4 v = df[i];
                v.x += dz[4 * i] + sDz[slot][4 * i];
                v.y += dz[4 * i + 1] + sDz[slot][4 * i + 1];
                v.z += dz[4 * i + 2] + sDz[slot][4 * i + 2];
                v.w += dz[4 * i + 3] + sDz[slot][4 * i + 3];
                df[i] = v;
            }
        }
        __syncthreads();
    }
}

// Weight pass: dW2 = dY^T H (block-diagonal), dW1 = dP^T Z, db2 = sum dY, db1 = sum dP over
// the selected anchors.  Split over anchors: each CTA stages chunks of kWChunk rows in shared
// memory (double-buffered bulk copies) and accumulates fixed output items in registers (4
// columns per item: 2 shared loads per 4 FMAs); its totals go to its partial row, summed
// across CTAs in a fixed order.
constexpr int kWThreads = 256;
constexpr int kWChunk = 32;
constexpr int kItemsW2 = kNOut * (kH / 4);                // 880
constexpr int kItemsW1 = 3 * kH * (kDin / 4);             // 864
constexpr int kItems4 = kItemsW2 + kItemsW1;              // 1744
constexpr int kPerThread4 = (kItems4 + kWThreads - 1) / kWThreads;   // 7
constexpr int kItems1 = kNOut + kNB1;                     // 206 bias sums

// Shared-memory stage of one chunk: the four row arrays back to back, each [kWChunk][row].
constexpr int kWStageFloats = kWChunk * (kRowY + kRowH + kRowP + kRowZ);
constexpr int kWSmemBytes = 2 * kWStageFloats * (int)sizeof(float);
constexpr uint32_t kWWaitLimit = 1u << 24;

// Bulk copies of chunk ch's rows (the first nv of them; every row is a multiple of 16 bytes and
// the arrays start 256-byte aligned) into stage `st`, completing on mbar.
__device__ __forceinline__ void weights_issue(const DbArgs& a, float* stage, uint32_t ch,
                                              uint32_t M, uint64_t* mbar) {
    const uint32_t r0 = ch * kWChunk;
    const uint32_t nv = min((uint32_t)kWChunk, M - r0);
    tc::mbar_expect_tx(mbar, nv * 4u * (kRowY + kRowH + kRowP + kRowZ));
    tc::bulk_load(stage, a.rowY + (size_t)r0 * kRowY, nv * 4u * kRowY, mbar);
    tc::bulk_load(stage + kWChunk * kRowY, a.rowH + (size_t)r0 * kRowH, nv * 4u * kRowH, mbar);
    tc::bulk_load(stage + kWChunk * (kRowY + kRowH), a.rowP + (size_t)r0 * kRowP,
                  nv * 4u * kRowP, mbar);
    tc::bulk_load(stage + kWChunk * (kRowY + kRowH + kRowP), a.rowZ + (size_t)r0 * kRowZ,
                  nv * 4u * kRowZ, mbar);
}

// The chunks arrive by bulk copies into two shared-memory stages: the copy of a CTA's next
// chunk is issued before its current one is summed (the other stage was released by the
// barrier that ended the previous chunk), so the CTA's loads overlap its arithmetic.
__global__ void __launch_bounds__(kWThreads) decode_bwd_weights(DbArgs a) {
    extern __shared__ __align__(16) float s_w[];
    __shared__ __align__(8) uint64_t mbar[2];
    const uint32_t M = a.counts->n_selected;
    const int t = threadIdx.x;
    float4 acc[kPerThread4];
#pragma unroll
    for (int q = 0; q < kPerThread4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    float acc1 = 0.f;
    const uint32_t nchunks = (M + kWChunk - 1) / kWChunk;
    if (t == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        if (blockIdx.x < nchunks) weights_issue(a, s_w, blockIdx.x, M, &mbar[0]);
    }
    __syncthreads();
    bool timed_out = false;
    uint32_t i = 0;
    for (uint32_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x, ++i) {
        const uint32_t st = i & 1u;
        float* stage = s_w + st * kWStageFloats;
        if (t == 0 && ch + gridDim.x < nchunks)
            weights_issue(a, s_w + (st ^ 1u) * kWStageFloats, ch + gridDim.x, M, &mbar[st ^ 1u]);
        if (!tc::mbar_wait(&mbar[st], (i >> 1) & 1u, kWWaitLimit)) {
            timed_out = true;
            // the copies may still be landing: wait for them (bounded) before moving on
            tc::mbar_wait(&mbar[st], (i >> 1) & 1u, kWWaitLimit);
        }
        const int nv = (int)min((uint32_t)kWChunk, M - ch * kWChunk);
        float(*sY)[kRowY] = reinterpret_cast<float(*)[kRowY]>(stage);
        float(*sH)[kRowH] = reinterpret_cast<float(*)[kRowH]>(stage + kWChunk * kRowY);
        float(*sP)[kRowP] = reinterpret_cast<float(*)[kRowP]>(stage + kWChunk * (kRowY + kRowH));
        float(*sZ)[kRowZ] =
            reinterpret_cast<float(*)[kRowZ]>(stage + kWChunk * (kRowY + kRowH + kRowP));
        if (nv < kWChunk) {                   // the last, partial chunk: zero the rows past it
            for (int e = t; e < (kWChunk - nv) * kRowY; e += kWThreads) sY[nv + e / kRowY][e % kRowY] = 0.f;
            for (int e = t; e < (kWChunk - nv) * kRowH; e += kWThreads) {
                sH[nv + e / kRowH][e % kRowH] = 0.f;
                sP[nv + e / kRowP][e % kRowP] = 0.f;
            }
            for (int e = t; e < (kWChunk - nv) * kRowZ; e += kWThreads) sZ[nv + e / kRowZ][e % kRowZ] = 0.f;
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < kPerThread4; ++q) {
            const int item = t + q * kWThreads;
            if (item < kItemsW2) {
                const int row = item / (kH / 4), c4 = item % (kH / 4);
                const int hc = dec_of(row) * kH + 4 * c4;
                float4 s = acc[q];
#pragma unroll 8
                for (int k = 0; k < kWChunk; ++k) {
                    const float yv = sY[k][row];
                    const float4 hv = *reinterpret_cast<const float4*>(&sH[k][hc]);
                    s.x = fmaf(yv, hv.x, s.x); s.y = fmaf(yv, hv.y, s.y);
                    s.z = fmaf(yv, hv.z, s.z); s.w = fmaf(yv, hv.w, s.w);
                }
                acc[q] = s;
            } else if (item < kItems4) {
                const int it = item - kItemsW2;
                const int row = it / (kDin / 4), c4 = it % (kDin / 4);
                float4 s = acc[q];
#pragma unroll 8
                for (int k = 0; k < kWChunk; ++k) {
                    const float pv = sP[k][row];
                    const float4 zv = *reinterpret_cast<const float4*>(&sZ[k][4 * c4]);
                    s.x = fmaf(pv, zv.x, s.x); s.y = fmaf(pv, zv.y, s.y);
                    s.z = fmaf(pv, zv.z, s.z); s.w = fmaf(pv, zv.w, s.w);
                }
                acc[q] = s;
            }
        }
        if (t < kItems1) {
            float s = 0.f;
            if (t < kNOut) {
                for (int k = 0; k < kWChunk; ++k) s += sY[k][t];
            } else {
                for (int k = 0; k < kWChunk; ++k) s += sP[k][t - kNOut];
            }
            acc1 += s;
        }
        __syncthreads();                      // this stage is free for the copy after next
    }
    if (timed_out && t == 0) atomicExch(const_cast<uint32_t*>(&a.counts->timeout), 1u);
    // this CTA's totals -> its partial row (flat layout of the decoder gradients)
    float* out = a.partial + (size_t)blockIdx.x * kNWeights;
#pragma unroll
    for (int q = 0; q < kPerThread4; ++q) {
        const int item = t + q * kWThreads;
        const float v4[4] = {acc[q].x, acc[q].y, acc[q].z, acc[q].w};
        if (item < kItemsW2) {
            const int row = item / (kH / 4), c4 = item % (kH / 4);
#pragma unroll
            for (int e = 0; e < 4; ++e) out[kOffW2 + row * kH + 4 * c4 + e] = v4[e];
        } else if (item < kItems4) {
            const int it = item - kItemsW2;
            const int row = it / (kDin / 4), c4 = it % (kDin / 4);
#pragma unroll
            for (int e = 0; e < 4; ++e) out[row * kDin + 4 * c4 + e] = v4[e];
        }
    }
    if (t < kItems1) {
        if (t < kNOut) out[kOffB2 + t] = acc1;
        else out[kOffB1 + (t - kNOut)] = acc1;
    }
}

// Appearance weight gradients (Sec. 4.4): dWa[o][c] = sum over the selected anchors of the
// colour decoder's pre-activation gradient dp_o (rowP columns 32..63) times the anchor's code
// value c.  Thread (o, c) of each CTA accumulates over chunks of kWChunk rows staged in shared
// memory; its total goes to the CTA's partial row, summed across CTAs by reduce_app in a
// fixed order.
static_assert(kWChunk * kMaxApp == kAppItems, "one code value staged per thread");

__global__ void __launch_bounds__(kAppItems) decode_bwd_app_weights(DbArgs a,
                                                                    float* __restrict__ part) {
    __shared__ float sP[kWChunk][kH + 1];
    __shared__ float sC[kWChunk][kMaxApp];
    const uint32_t M = a.counts->n_selected;
    const int t = threadIdx.x, o = t / kMaxApp, q = t % kMaxApp;
    const int napp = a.mlp.A;
    float acc = 0.f;
    const uint32_t nchunks = (M + kWChunk - 1) / kWChunk;
    for (uint32_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const uint32_t r0 = ch * kWChunk;
        const int nv = (int)min((uint32_t)kWChunk, M - r0);
        __syncthreads();
        for (int e = t; e < kWChunk * kH; e += kAppItems) {
            const int k = e / kH, h = e % kH;
            sP[k][h] = k < nv ? a.rowP[(size_t)(r0 + k) * kRowP + kH + h] : 0.f;
        }
        {
            const int k = t / kMaxApp, c = t % kMaxApp;
            sC[k][c] = (k < nv && c < napp) ? a.mlp.app[(size_t)a.sel_idx[r0 + k] * napp + c] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kWChunk; ++k) acc = fmaf(sP[k][o], sC[k][q], acc);
    }
    part[(size_t)blockIdx.x * kAppItems + t] = acc;
}

// dw1_app[o][c] += sum over blocks of part[b][o * kMaxApp + c] (fixed order, c < A).
__global__ void __launch_bounds__(kAppItems) reduce_app(const float* __restrict__ part,
                                                        int nblocks, float* dw1_app, int napp) {
    const int t = threadIdx.x, o = t / kMaxApp, q = t % kMaxApp;
    float s = 0.f;
#pragma unroll 8
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * kAppItems + t];
    if (q < napp) dw1_app[o * napp + q] += s;
}

// dmlp[e] += sum over blocks of partial[b][e].  A CTA owns 32 consecutive outputs (one per
// lane, coalesced reads); its 8 warps sum interleaved blocks, then warp 0 adds the 8 warp
// sums in a fixed order: deterministic.
constexpr int kRedWarps = 8;

__device__ __forceinline__ float* grad_slot(const ogs_mlp& grads, int e) {
    int i = e;
    if (i < kNW1) return const_cast<float*>(grads.w1) + i;
    if ((i -= kNW1) < kNB1) return const_cast<float*>(grads.b1) + i;
    if ((i -= kNB1) < kK * kH) return const_cast<float*>(grads.w2_op) + i;
    if ((i -= kK * kH) < 3 * kK * kH) return const_cast<float*>(grads.w2_col) + i;
    if ((i -= 3 * kK * kH) < 7 * kK * kH) return const_cast<float*>(grads.w2_cov) + i;
    if ((i -= 7 * kK * kH) < kK) return const_cast<float*>(grads.b2_op) + i;
    if ((i -= kK) < 3 * kK) return const_cast<float*>(grads.b2_col) + i;
    return const_cast<float*>(grads.b2_cov) + (i - 3 * kK);
}

__global__ void __launch_bounds__(32 * kRedWarps) reduce_partials(const float* __restrict__ partial,
                                                                  int nblocks, ogs_mlp grads) {
    __shared__ float s[kRedWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    float acc = 0.f;
    if (e < kNWeights) {
#pragma unroll 4
        for (int b = warp; b < nblocks; b += kRedWarps) acc += partial[(size_t)b * kNWeights + e];
    }
    s[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && e < kNWeights) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < kRedWarps; ++w) t += s[w][lane];
        *grad_slot(grads, e) += t;
    }
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

// x *= *s (the chain-rule factor that a loss's backward receives)
__global__ void scale_kernel(float* __restrict__ x, int64_t n, const float* __restrict__ s) {
    const float f = *s;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= f;
}

// One parameter: m, v moments; step lr * m_hat / (sqrt(v_hat) + eps) with the bias
// corrections folded into reciprocals (ibc1 = 1/(1 - b1^t), ibc2 = 1/(1 - b2^t)) and one
// fast division, so the update costs a handful of instructions and the kernel stays
// memory-bound.
__device__ __forceinline__ void adam_one(float& p, float& g, float& m, float& v, float lr,
                                         float b1, float b2, float eps, float ibc1, float ibc2,
                                         int zero_grad) {
    m = fmaf(b1, m, (1.f - b1) * g);
    v = fmaf(b2, v, (1.f - b2) * g * g);
    p -= __fdividef(lr * ibc1 * m, __fsqrt_rn(v * ibc2) + eps);
    if (zero_grad) g = 0.f;
}

// Streaming update: 16-byte vectors when all four arrays are 16-byte aligned (n/4 vectors
// plus a scalar tail), scalars otherwise.  HBM-bound: 16 B read + 12 B written per parameter
// (+4 B for the gradients that were nonzero, cleared with zero_grad).
__global__ void __launch_bounds__(256) adam_kernel(float* __restrict__ p, float* __restrict__ grad,
                                                   float* __restrict__ m, float* __restrict__ v,
                                                   int64_t n, float lr, float b1, float b2,
                                                   float eps, float ibc1, float ibc2,
                                                   int zero_grad, int vec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t first = 0;
    if (vec) {
        const int64_t n4 = n / 4;
        float4* p4 = reinterpret_cast<float4*>(p);
        float4* g4 = reinterpret_cast<float4*>(grad);
        float4* m4 = reinterpret_cast<float4*>(m);
        float4* v4 = reinterpret_cast<float4*>(v);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            float4 P = p4[i], G = g4[i], M = m4[i], V = v4[i];
            // most anchors get no gradient in a step: clear only vectors that hold one
            const bool touched = G.x != 0.f || G.y != 0.f || G.z != 0.f || G.w != 0.f;
            adam_one(P.x, G.x, M.x, V.x, lr, b1, b2, eps, ibc1, ibc2, zero_grad);
            adam_one(P.y, G.y, M.y, V.y, lr, b1, b2, eps, ibc1, ibc2, zero_grad);
            adam_one(P.z, G.z, M.z, V.z, lr, b1, b2, eps, ibc1, ibc2, zero_grad);
            adam_one(P.w, G.w, M.w, V.w, lr, b1, b2, eps, ibc1, ibc2, zero_grad);
            p4[i] = P; m4[i] = M; v4[i] = V;
            if (zero_grad && touched) g4[i] = G;
        }
        first = 4 * n4;
    }
    for (int64_t i = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float P = p[i], G = grad[i], M = m[i], V = v[i];
        adam_one(P, G, M, V, lr, b1, b2, eps, ibc1, ibc2, zero_grad);
        p[i] = P; m[i] = M; v[i] = V;
        if (zero_grad) grad[i] = G;
    }
}

}  // namespace

cudaError_t db::launch_weight_pass(const DbArgs& a, const DbScratch& s, const ogs_mlp& dmlp,
                                   cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(decode_bwd_weights,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmemBytes);
    if (e != cudaSuccess) return e;
    decode_bwd_weights<<<kDbBlocks, kWThreads, kWSmemBytes, st>>>(a);
    reduce_partials<<<(kNWeights + 31) / 32, 32 * kRedWarps, 0, st>>>(s.partial, kDbBlocks, dmlp);
    if (a.mlp.A > 0) {
        decode_bwd_app_weights<<<kDbBlocks, kAppItems, 0, st>>>(a, s.partial_app);
        reduce_app<<<1, kAppItems, 0, st>>>(s.partial_app, kDbBlocks,
                                            const_cast<float*>(dmlp.w1_app), a.mlp.A);
    }
    return cudaGetLastError();
}

}  // namespace ogs

using namespace ogs;
using namespace ogs::db;

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

extern "C" size_t ogs_decode_bwd_scratch_bytes(int64_t sel_cap) {
    return db_layout(sel_cap < 0 ? 0 : sel_cap, nullptr, nullptr);
}

extern "C" ogs_status ogs_decode_bwd(const float* pos, const float* feat, const float* offs,
                                     const float* lv, int64_t N, const ogs_mlp* mlp,
                                     const ogs_camera* cam, const uint32_t* sel_idx,
                                     const float* sel_w, int64_t sel_cap,
                                     const ogs_counts* counts, const float* dmeans,
                                     const float* dscales, const float* dquats, const float* drec,
                                     float* dfeat, float* doffs, float* dlv, const ogs_mlp* dmlp,
                                     void* scratch, size_t scratch_bytes, void* stream) {
    if (!pos || !feat || !offs || !lv || !mlp || !cam || !sel_idx || !sel_w || !counts ||
        !dmeans || !dscales || !dquats || !drec || !dfeat || !doffs || !dlv || !dmlp || !scratch)
        return OGS_ERR_ARG;
    if (mlp->F != kF || mlp->H != kH || mlp->k != kK || N < 0 || sel_cap < 0 || !app_ok(*mlp))
        return OGS_ERR_ARG;
    if (!dmlp->w1 || !dmlp->b1 || !dmlp->w2_op || !dmlp->b2_op || !dmlp->w2_col ||
        !dmlp->b2_col || !dmlp->w2_cov || !dmlp->b2_cov)
        return OGS_ERR_ARG;
    if (mlp->A > 0 && (!dmlp->w1_app || !dmlp->app)) return OGS_ERR_ARG;
    if (scratch_bytes < ogs_decode_bwd_scratch_bytes(sel_cap) || !aligned(scratch, 16) ||
        !aligned(dquats, 16) || !aligned(feat, 16) || !aligned(dfeat, 16))
        return OGS_ERR_ARG;
    if (sel_cap == 0) return OGS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    DbScratch sc;
    db_layout(sel_cap, scratch, &sc);
    DbArgs a{pos, feat, offs, lv, sel_idx, sel_w, counts, *mlp, make_cam(*cam), dmeans, dscales,
             dquats, drec, dfeat, doffs, dlv, sc.rowY, sc.rowH, sc.rowP, sc.rowZ, sc.partial,
             const_cast<float*>(dmlp->app)};
    if (mlp->A > 0)
        decode_bwd_rows<true><<<stride_grid(sel_cap, kRowAnchors, 3), kDbThreads, 0, st>>>(a);
    else
        decode_bwd_rows<false><<<stride_grid(sel_cap, kRowAnchors, 3), kDbThreads, 0, st>>>(a);
    if (launch_weight_pass(a, sc, *dmlp, st) != cudaSuccess) return OGS_ERR_CUDA;
    return launch_status();
}

extern "C" ogs_status ogs_loss_l1(const float* img, const float* target, int64_t n, float* dimg,
                                  float* loss, void* stream) {
    if (!img || !target || !dimg || n <= 0) return OGS_ERR_ARG;
    l1_kernel<<<stride_grid(n, 256, 8), 256, 0, (cudaStream_t)stream>>>(img, target, n,
                                                                         1.0f / (float)n, dimg, loss);
    return launch_status();
}

// Adam over the rows whose stamp equals `value` (the anchors a training step selected).  A
// warp takes 32 rows at a time: their stamps are read in one coalesced load, and the warp then
// walks the touched ones, its lanes covering a row's elements (rows of up to 64 values in two
// rounds, longer rows in more); gradients of updated rows are cleared.
__global__ void __launch_bounds__(256) adam_rows_kernel(float* __restrict__ p,
                                                        float* __restrict__ grad,
                                                        float* __restrict__ m,
                                                        float* __restrict__ v, int64_t rows,
                                                        int row_len,
                                                        const uint32_t* __restrict__ stamp,
                                                        uint32_t value, float lr, float b1,
                                                        float b2, float eps, float ibc1,
                                                        float ibc2, int zero_grad) {
    const int lane = (int)lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = warp * 32; r0 < rows; r0 += nwarps * 32) {
        const int64_t r = r0 + lane;
        const bool hit = r < rows && stamp[r] == value;
        uint32_t todo = __ballot_sync(0xffffffffu, hit);
        while (todo) {
            const int b = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t base = (r0 + b) * (int64_t)row_len;
            for (int e = lane; e < row_len; e += 32) {
                float P = p[base + e], G = grad[base + e], M = m[base + e], V = v[base + e];
                adam_one(P, G, M, V, lr, b1, b2, eps, ibc1, ibc2, zero_grad);
                p[base + e] = P;
                m[base + e] = M;
                v[base + e] = V;
                if (zero_grad) grad[base + e] = G;
            }
        }
    }
}

// stamp[sel_idx[r]] = value for the r < counts->n_selected selected anchors
__global__ void stamp_rows_kernel(const uint32_t* __restrict__ sel_idx,
                                  const ogs_counts* __restrict__ counts,
                                  uint32_t* __restrict__ stamp, uint32_t value) {
    const uint32_t M = counts->n_selected;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < M; r += gridDim.x * blockDim.x)
        stamp[sel_idx[r]] = value;
}

extern "C" ogs_status ogs_stamp_selected(const uint32_t* sel_idx, const ogs_counts* counts,
                                         int64_t sel_cap, uint32_t* stamp, uint32_t value,
                                         void* stream) {
    if (!sel_idx || !counts || !stamp || sel_cap < 0) return OGS_ERR_ARG;
    if (sel_cap == 0) return OGS_OK;
    stamp_rows_kernel<<<stride_grid(sel_cap, 256, 8), 256, 0, (cudaStream_t)stream>>>(
        sel_idx, counts, stamp, value);
    return launch_status();
}

extern "C" ogs_status ogs_adam_rows(float* param, float* grad, float* m, float* v, int64_t rows,
                                    int32_t row_len, const uint32_t* stamp, uint32_t value,
                                    float lr, float beta1, float beta2, float eps, int32_t step,
                                    int32_t zero_grad, void* stream) {
    if (!param || !grad || !m || !v || !stamp || rows < 0 || row_len < 1 || step < 1)
        return OGS_ERR_ARG;
    if (rows == 0) return OGS_OK;
    const double bc1 = 1.0 - pow((double)beta1, (double)step);
    const double bc2 = 1.0 - pow((double)beta2, (double)step);
    adam_rows_kernel<<<stride_grid((rows + 31) / 32 * 32, 256, 8), 256, 0,
                       (cudaStream_t)stream>>>(param, grad, m, v, rows, row_len, stamp, value,
                                               lr, beta1, beta2, eps, (float)(1.0 / bc1),
                                               (float)(1.0 / bc2), zero_grad);
    return launch_status();
}

// flag |= bit if any of x[0..n) is NaN or infinite (one atomic per warp that finds one)
__global__ void nonfinite_kernel(const float* __restrict__ x, int64_t n, uint32_t* flag,
                                 uint32_t bit) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(flag, bit);
}

extern "C" ogs_status ogs_scan_nonfinite(const float* x, int64_t n, uint32_t* flag, uint32_t bit,
                                         void* stream) {
    if (!x || !flag || n < 0 || bit == 0) return OGS_ERR_ARG;
    if (n == 0) return OGS_OK;
    nonfinite_kernel<<<stride_grid(n, 256, 8), 256, 0, (cudaStream_t)stream>>>(x, n, flag, bit);
    return launch_status();
}

extern "C" ogs_status ogs_counts_status(const ogs_counts* counts, uint32_t nonfinite) {
    if (!counts) return OGS_ERR_ARG;
    if (nonfinite) return OGS_ERR_NONFINITE;
    if (counts->timeout) return OGS_ERR_TIMEOUT;
    if (counts->overflow) return OGS_ERR_CAPACITY;
    return OGS_OK;
}

extern "C" ogs_status ogs_scale(float* x, int64_t n, const float* s, void* stream) {
    if (!x || !s || n < 0) return OGS_ERR_ARG;
    if (n == 0) return OGS_OK;
    scale_kernel<<<stride_grid(n, 256, 8), 256, 0, (cudaStream_t)stream>>>(x, n, s);
    return launch_status();
}

extern "C" ogs_status ogs_adam(float* param, float* grad, float* m, float* v, int64_t n, float lr,
                               float beta1, float beta2, float eps, int32_t step,
                               int32_t zero_grad, void* stream) {
    if (!param || !grad || !m || !v || n < 0 || step < 1) return OGS_ERR_ARG;
    if (n == 0) return OGS_OK;
    const double bc1 = 1.0 - pow((double)beta1, (double)step);
    const double bc2 = 1.0 - pow((double)beta2, (double)step);
    const int vec = aligned(param, 16) && aligned(grad, 16) && aligned(m, 16) && aligned(v, 16);
    adam_kernel<<<stride_grid(vec ? n / 4 + 1 : n, 256, 8), 256, 0, (cudaStream_t)stream>>>(
        param, grad, m, v, n, lr, beta1, beta2, eps, (float)(1.0 / bc1), (float)(1.0 / bc2),
        zero_grad, vec);
    return launch_status();
}
