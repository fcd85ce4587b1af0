// Photometric loss of Sec. 5.1.5: (1 - lambda) L1 + lambda (1 - SSIM), lambda = 0.2, SSIM with
// an 11x11 Gaussian window (sigma 1.5, separable, zero padded) and the usual C1 = 0.01^2,
// C2 = 0.03^2 (Wang et al. 2004), and its gradient with respect to the rendered image.
//
// With m1 = G*x, m2 = G*x^2, m3 = G*(x y) and the SSIM map S = A1 A2 / (B1 B2) (A1 = 2 m1 my
// + C1, A2 = 2 (m3 - m1 my) + C2, B1 = m1^2 + my^2 + C1, B2 = m2 - m1^2 + sy^2 + C2):
//   dS/dm1 = S (2my/A1 - 2my/A2 - 2m1/B1 + 2m1/B2),  dS/dm2 = -S/B2,  dS/dm3 = 2S/A2,
// and for the mean SSIM:  d/dx = G*g1 + 2 x (G*g2) + y (G*g3), g_i = dS/dm_i / n.
// Two tiled passes (moments -> SSIM map and partial maps; blur of the partial maps ->
// gradient), each staging its tile and halo in shared memory; bound by FP32 instruction issue
// (11-tap blurs of every moment in both directions).  A training loop that renders against
// fixed targets can compute the target's two moments once (ogs_ssim_target_stats) and pass
// them in, so that the forward pass blurs three moments instead of five.
#include <cmath>

#include "internal.cuh"

namespace ogs {
namespace {

constexpr int kWin = 11;
constexpr int kRad = kWin / 2;
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct Win {
    float w[kWin];
};

Win make_window() {
    Win g;
    double s = 0.0, t[kWin];
    for (int i = 0; i < kWin; ++i) {
        const double x = i - kRad;
        t[i] = std::exp(-x * x / (2.0 * 1.5 * 1.5));
        s += t[i];
    }
    for (int i = 0; i < kWin; ++i) g.w[i] = (float)(t[i] / s);
    return g;
}

// Tiled passes: a CTA owns a kTX x kTY output tile of one channel.  It stages the inputs of
// the tile plus a kRad halo in shared memory (zero outside the image: the zero-padded window),
// blurs horizontally into shared memory and vertically into registers.
constexpr int kTX = 32, kTY = 32;
constexpr int kHX = kTX + 2 * kRad, kHY = kTY + 2 * kRad;   // 42 x 42 staged inputs
constexpr int kLossThreads = 256;

__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane_id() == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < kLossThreads / 32; ++i) s += red[i];
    return s;                                       // valid in thread 0
}

// Register-blocked 11-tap blurs: a thread produces kRun consecutive outputs along the blur
// direction from kRun + 10 loaded inputs (each input loaded once instead of once per tap).
constexpr int kRun = 4;
constexpr int kSpan = kRun + kWin - 1;                     // 14 inputs per run
constexpr int kHRuns = kHY * (kTX / kRun);                 // 42 rows x 8 runs = 336
constexpr int kVRuns = kTX * (kTY / kRun);                 // 32 columns x 8 runs = 256

// pass 1: the blurred moments -> SSIM map (summed) and the three partial maps
// gp_i = dS/dm_i / n for the backward.  The five moments are G*x, G*y, G*x^2, G*y^2, G*xy;
// with kCached the target's two (G*y, G*y^2) come precomputed in ystat[2][C][H][W] (they do
// not change between training steps) and only three are blurred here.
template <bool kCached>
__global__ void __launch_bounds__(kLossThreads) ssim_fwd(const float* __restrict__ x,
                                                         const float* __restrict__ y, int H, int W,
                                                         Win g, float inv_n,
                                                         float* __restrict__ gp, int64_t n,
                                                         float* __restrict__ ssim_sum,
                                                         const float* __restrict__ ystat) {
    constexpr int kM = kCached ? 3 : 5;           // moments blurred here: x, [y], x^2, [y^2], xy
    __shared__ float sx[kHY][kHX + 1];
    __shared__ float sy[kHY][kHX + 1];
    __shared__ float hs[kM][kHY][kTX + 1];
    __shared__ float red[kLossThreads / 32];
    const int c = blockIdx.z;
    const int x0 = blockIdx.x * kTX - kRad, y0 = blockIdx.y * kTY - kRad;
    const int64_t plane = (int64_t)c * H * W;
    {
        // 6 rows of 42 per pass, 7 passes; all loads issued before any store (threads 252..255
        // idle)
        constexpr int kRowsPer = kLossThreads / kHX, kPasses = (kHY + kRowsPer - 1) / kRowsPer;
        const int q = threadIdx.x % kHX, r0 = threadIdx.x / kHX;
        const bool act = threadIdx.x < kRowsPer * kHX;
        float vx[kPasses], vy[kPasses];
#pragma unroll
        for (int k = 0; k < kPasses; ++k) {
            const int gy = y0 + r0 + kRowsPer * k, gx = x0 + q;
            const bool in = act && r0 + kRowsPer * k < kHY && gx >= 0 && gx < W && gy >= 0 && gy < H;
            const int64_t i = plane + (int64_t)gy * W + gx;
            vx[k] = in ? x[i] : 0.f;
            vy[k] = in ? y[i] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kPasses; ++k) {
            if (act && r0 + kRowsPer * k < kHY) {
                sx[r0 + kRowsPer * k][q] = vx[k];
                sy[r0 + kRowsPer * k][q] = vy[k];
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kHRuns; e += kLossThreads) {
        const int r = e >> 3, q0 = (e & 7) * kRun;
        float u[kSpan], v[kSpan];
#pragma unroll
        for (int k = 0; k < kSpan; ++k) { u[k] = sx[r][q0 + k]; v[k] = sy[r][q0 + k]; }
        float acc[kM][kRun];
#pragma unroll
        for (int t = 0; t < kRun; ++t)
#pragma unroll
            for (int j = 0; j < kM; ++j) acc[j][t] = 0.f;
#pragma unroll
        for (int k = 0; k < kSpan; ++k) {
            // channel order: x, x^2, xy (cached) or x, y, x^2, y^2, xy
            float ch[kM];
            if (kCached) {
                ch[0] = u[k];
                ch[1] = u[k] * u[k];
                ch[kM - 1] = u[k] * v[k];
            } else {
                ch[0] = u[k];
                ch[1] = v[k];
                ch[2] = u[k] * u[k];
                ch[3] = v[k] * v[k];
                ch[kM - 1] = u[k] * v[k];
            }
#pragma unroll
            for (int t = 0; t < kRun; ++t) {
                const int tap = k - t;
                if (tap < 0 || tap >= kWin) continue;
                const float w = g.w[tap];
#pragma unroll
                for (int j = 0; j < kM; ++j) acc[j][t] = fmaf(w, ch[j], acc[j][t]);
            }
        }
#pragma unroll
        for (int t = 0; t < kRun; ++t)
#pragma unroll
            for (int j = 0; j < kM; ++j) hs[j][r][q0 + t] = acc[j][t];
    }
    __syncthreads();
    float local = 0.f;
    {
        const int qc = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * kRun;   // one run per thread
        float m[kM][kRun];
#pragma unroll
        for (int t = 0; t < kRun; ++t)
#pragma unroll
            for (int j = 0; j < kM; ++j) m[j][t] = 0.f;
#pragma unroll
        for (int k = 0; k < kSpan; ++k) {
            float hv[kM];
#pragma unroll
            for (int j = 0; j < kM; ++j) hv[j] = hs[j][r0 + k][qc];
#pragma unroll
            for (int t = 0; t < kRun; ++t) {
                const int tap = k - t;
                if (tap < 0 || tap >= kWin) continue;
                const float w = g.w[tap];
#pragma unroll
                for (int j = 0; j < kM; ++j) m[j][t] = fmaf(w, hv[j], m[j][t]);
            }
        }
        const int gx = x0 + kRad + qc;
#pragma unroll
        for (int t = 0; t < kRun; ++t) {
            const int gy = y0 + kRad + r0 + t;
            if (gx >= W || gy >= H) continue;
            const int64_t i = plane + (int64_t)gy * W + gx;
            float mx, my, exx, eyy, exy;
            if (kCached) {
                mx = m[0][t]; exx = m[1][t]; exy = m[2][t];
                my = ystat[i]; eyy = ystat[n + i];
            } else {
                mx = m[0][t]; my = m[1][t]; exx = m[2][t]; eyy = m[3][t]; exy = m[4][t];
            }
            const float vx = exx - mx * mx, vy = eyy - my * my, vxy = exy - mx * my;
            const float A1 = 2.f * mx * my + kC1, A2 = 2.f * vxy + kC2;
            const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
            // four fast reciprocals (a few ulp) in place of seven divisions: the epilogue
            // would otherwise cost as much as the blurs
            const float iA1 = __fdividef(1.f, A1), iA2 = __fdividef(1.f, A2);
            const float iB1 = __fdividef(1.f, B1), iB2 = __fdividef(1.f, B2);
            const float S = A1 * A2 * iB1 * iB2;
            local += S;
            const float sS = S * inv_n;
            gp[i] = 2.f * sS * (my * (iA1 - iA2) + mx * (iB2 - iB1));
            gp[n + i] = -sS * iB2;
            gp[2 * n + i] = 2.f * sS * iA2;
        }
    }
    const float s = block_sum(local, red);
    if (threadIdx.x == 0) atomicAdd(ssim_sum, s);
}

// pass 2: blur of the partial maps -> dSSIM/dx = G*gp0 + 2 x (G*gp1) + y (G*gp2);
// dimg = (1 - lam) sign(x - y) / n - lam dSSIM/dx, and the L1 sum
__global__ void __launch_bounds__(kLossThreads) ssim_bwd(const float* __restrict__ gp,
                                                         const float* __restrict__ x,
                                                         const float* __restrict__ y, int H, int W,
                                                         Win g, float lam, float inv_n, int64_t n,
                                                         float* __restrict__ dimg,
                                                         float* __restrict__ l1_sum) {
    __shared__ float sg[3][kHY][kHX + 1];
    __shared__ float hs[3][kHY][kTX + 1];
    __shared__ float red[kLossThreads / 32];
    const int c = blockIdx.z;
    const int x0 = blockIdx.x * kTX - kRad, y0 = blockIdx.y * kTY - kRad;
    const int64_t plane = (int64_t)c * H * W;
    {
        constexpr int kRowsPer = kLossThreads / kHX, kPasses = (kHY + kRowsPer - 1) / kRowsPer;
        const int q = threadIdx.x % kHX, r0 = threadIdx.x / kHX;
        const bool act = threadIdx.x < kRowsPer * kHX;
        float v0[kPasses], v1[kPasses], v2[kPasses];
#pragma unroll
        for (int k = 0; k < kPasses; ++k) {
            const int gy = y0 + r0 + kRowsPer * k, gx = x0 + q;
            const bool in = act && r0 + kRowsPer * k < kHY && gx >= 0 && gx < W && gy >= 0 && gy < H;
            const int64_t i = plane + (int64_t)gy * W + gx;
            v0[k] = in ? gp[i] : 0.f;
            v1[k] = in ? gp[n + i] : 0.f;
            v2[k] = in ? gp[2 * n + i] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kPasses; ++k) {
            if (act && r0 + kRowsPer * k < kHY) {
                sg[0][r0 + kRowsPer * k][q] = v0[k];
                sg[1][r0 + kRowsPer * k][q] = v1[k];
                sg[2][r0 + kRowsPer * k][q] = v2[k];
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kHRuns; e += kLossThreads) {
        const int r = e >> 3, q0 = (e & 7) * kRun;
        float acc[3][kRun];
#pragma unroll
        for (int t = 0; t < kRun; ++t)
#pragma unroll
            for (int j = 0; j < 3; ++j) acc[j][t] = 0.f;
#pragma unroll
        for (int k = 0; k < kSpan; ++k) {
            float gv[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) gv[j] = sg[j][r][q0 + k];
#pragma unroll
            for (int t = 0; t < kRun; ++t) {
                const int tap = k - t;
                if (tap < 0 || tap >= kWin) continue;
                const float w = g.w[tap];
#pragma unroll
                for (int j = 0; j < 3; ++j) acc[j][t] = fmaf(w, gv[j], acc[j][t]);
            }
        }
#pragma unroll
        for (int t = 0; t < kRun; ++t)
#pragma unroll
            for (int j = 0; j < 3; ++j) hs[j][r][q0 + t] = acc[j][t];
    }
    __syncthreads();
    float local = 0.f;
    {
        const int qc = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * kRun;
        const int gx = x0 + kRad + qc;
        float xs[kRun], ys[kRun];                 // loaded before the blur, used after it
#pragma unroll
        for (int t = 0; t < kRun; ++t) {
            const int gy = y0 + kRad + r0 + t;
            const bool in = gx < W && gy < H;
            const int64_t i = plane + (int64_t)gy * W + gx;
            xs[t] = in ? x[i] : 0.f;
            ys[t] = in ? y[i] : 0.f;
        }
        float m[3][kRun];
#pragma unroll
        for (int t = 0; t < kRun; ++t)
#pragma unroll
            for (int j = 0; j < 3; ++j) m[j][t] = 0.f;
#pragma unroll
        for (int k = 0; k < kSpan; ++k) {
            float hv[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) hv[j] = hs[j][r0 + k][qc];
#pragma unroll
            for (int t = 0; t < kRun; ++t) {
                const int tap = k - t;
                if (tap < 0 || tap >= kWin) continue;
                const float w = g.w[tap];
#pragma unroll
                for (int j = 0; j < 3; ++j) m[j][t] = fmaf(w, hv[j], m[j][t]);
            }
        }
#pragma unroll
        for (int t = 0; t < kRun; ++t) {
            const int gy = y0 + kRad + r0 + t;
            if (gx >= W || gy >= H) continue;
            const int64_t i = plane + (int64_t)gy * W + gx;
            const float xi = xs[t], yi = ys[t];
            const float dssim = m[0][t] + 2.f * xi * m[1][t] + yi * m[2][t];
            const float df = xi - yi;
            local += fabsf(df);
            const float sgn = df > 0.f ? inv_n : (df < 0.f ? -inv_n : 0.f);
            dimg[i] = (1.f - lam) * sgn - lam * dssim;
        }
    }
    const float s = block_sum(local, red);
    if (threadIdx.x == 0) atomicAdd(l1_sum, s);
}

// The target's two window moments G*y and G*y^2 (zero padded), written to ystat[2][C][H][W]:
// the same tiling and blur order as ssim_fwd, so the cached form uses the same values.
__global__ void __launch_bounds__(kLossThreads) ssim_target_stats(const float* __restrict__ y,
                                                                  int H, int W, Win g, int64_t n,
                                                                  float* __restrict__ ystat) {
    __shared__ float sy[kHY][kHX + 1];
    __shared__ float hs[2][kHY][kTX + 1];
    const int c = blockIdx.z;
    const int x0 = blockIdx.x * kTX - kRad, y0 = blockIdx.y * kTY - kRad;
    const int64_t plane = (int64_t)c * H * W;
    for (int e = threadIdx.x; e < kHY * kHX; e += kLossThreads) {
        const int r = e / kHX, q = e % kHX;
        const int gy = y0 + r, gx = x0 + q;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        sy[r][q] = in ? y[plane + (int64_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kHRuns; e += kLossThreads) {
        const int r = e >> 3, q0 = (e & 7) * kRun;
        float acc[2][kRun];
#pragma unroll
        for (int t = 0; t < kRun; ++t) acc[0][t] = acc[1][t] = 0.f;
#pragma unroll
        for (int k = 0; k < kSpan; ++k) {
            const float v = sy[r][q0 + k], vv = v * v;
#pragma unroll
            for (int t = 0; t < kRun; ++t) {
                const int tap = k - t;
                if (tap < 0 || tap >= kWin) continue;
                acc[0][t] = fmaf(g.w[tap], v, acc[0][t]);
                acc[1][t] = fmaf(g.w[tap], vv, acc[1][t]);
            }
        }
#pragma unroll
        for (int t = 0; t < kRun; ++t) {
            hs[0][r][q0 + t] = acc[0][t];
            hs[1][r][q0 + t] = acc[1][t];
        }
    }
    __syncthreads();
    const int qc = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * kRun;
    float m[2][kRun];
#pragma unroll
    for (int t = 0; t < kRun; ++t) m[0][t] = m[1][t] = 0.f;
#pragma unroll
    for (int k = 0; k < kSpan; ++k) {
        const float h0 = hs[0][r0 + k][qc], h1 = hs[1][r0 + k][qc];
#pragma unroll
        for (int t = 0; t < kRun; ++t) {
            const int tap = k - t;
            if (tap < 0 || tap >= kWin) continue;
            m[0][t] = fmaf(g.w[tap], h0, m[0][t]);
            m[1][t] = fmaf(g.w[tap], h1, m[1][t]);
        }
    }
    const int gx = x0 + kRad + qc;
#pragma unroll
    for (int t = 0; t < kRun; ++t) {
        const int gy = y0 + kRad + r0 + t;
        if (gx >= W || gy >= H) continue;
        const int64_t i = plane + (int64_t)gy * W + gx;
        ystat[i] = m[0][t];
        ystat[n + i] = m[1][t];
    }
}

// loss = (1 - lam) * l1_sum / n + lam * (1 - ssim_sum / n), added to *loss
__global__ void combine_loss(const float* sums, int64_t n, float lam, float* loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0)
        *loss += (1.f - lam) * sums[1] / (float)n + lam * (1.f - sums[0] / (float)n);
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" size_t ogs_loss_l1_ssim_scratch_bytes(int32_t C, int32_t H, int32_t W) {
    return sizeof(float) * ((size_t)3 * C * H * W + 4) + 512;
}

extern "C" ogs_status ogs_ssim_target_stats(const float* target, int32_t C, int32_t H,
                                            int32_t W, float* ystat, void* stream) {
    if (!target || !ystat || C <= 0 || H <= 0 || W <= 0) return OGS_ERR_ARG;
    const dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY, C);
    ssim_target_stats<<<grid, kLossThreads, 0, (cudaStream_t)stream>>>(
        target, H, W, make_window(), (int64_t)C * H * W, ystat);
    return launch_status();
}

extern "C" ogs_status ogs_loss_l1_ssim(const float* img, const float* target, int32_t C,
                                       int32_t H, int32_t W, float lambda, float* dimg,
                                       float* loss, const float* target_stats, void* scratch,
                                       size_t scratch_bytes, void* stream) {
    if (!img || !target || !dimg || !scratch || C <= 0 || H <= 0 || W <= 0) return OGS_ERR_ARG;
    if (!(lambda >= 0.f && lambda <= 1.f)) return OGS_ERR_ARG;
    if (scratch_bytes < ogs_loss_l1_ssim_scratch_bytes(C, H, W) || !aligned(scratch, 16))
        return OGS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)C * H * W;
    Carver cv(scratch);
    float* gp = cv.take<float>(3 * n);
    float* sums = cv.take<float>(4);
    const Win g = make_window();
    if (cudaMemsetAsync(sums, 0, 4 * sizeof(float), st) != cudaSuccess) return OGS_ERR_CUDA;
    const dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY, C);
    const float inv_n = 1.0f / (float)n;
    if (target_stats)
        ssim_fwd<true><<<grid, kLossThreads, 0, st>>>(img, target, H, W, g, inv_n, gp, n, sums,
                                                      target_stats);
    else
        ssim_fwd<false><<<grid, kLossThreads, 0, st>>>(img, target, H, W, g, inv_n, gp, n, sums,
                                                       nullptr);
    ssim_bwd<<<grid, kLossThreads, 0, st>>>(gp, img, target, H, W, g, lambda, inv_n, n, dimg,
                                            sums + 1);
    if (loss) combine_loss<<<1, 32, 0, st>>>(sums, n, lambda, loss);
    return launch_status();
}
