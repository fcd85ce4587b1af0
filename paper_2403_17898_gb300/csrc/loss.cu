// Photometric loss of Sec. 5.1.5: (1 - lambda) L1 + lambda (1 - SSIM), lambda = 0.2, SSIM with
// an 11x11 Gaussian window (sigma 1.5, separable, zero padded) and the usual C1 = 0.01^2,
// C2 = 0.03^2 (Wang et al. 2004), and its gradient with respect to the rendered image.
//
// With m1 = G*x, m2 = G*x^2, m3 = G*(x y) and the SSIM map S = A1 A2 / (B1 B2) (A1 = 2 m1 my
// + C1, A2 = 2 (m3 - m1 my) + C2, B1 = m1^2 + my^2 + C1, B2 = m2 - m1^2 + sy^2 + C2):
//   dS/dm1 = S (2my/A1 - 2my/A2 - 2m1/B1 + 2m1/B2),  dS/dm2 = -S/B2,  dS/dm3 = 2S/A2,
// and for the mean SSIM:  d/dx = G*g1 + 2 x (G*g2) + y (G*g3), g_i = dS/dm_i / n.
// Four streaming passes (horizontal blur of 5 maps, vertical blur + SSIM map, horizontal blur
// of the 3 partial maps, vertical blur + gradient), all HBM-bound.
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

// horizontal blur of x, y, x^2, y^2, x y  ->  h[5][C*H*W]
__global__ void ssim_h5(const float* __restrict__ x, const float* __restrict__ y, int C, int H,
                        int W, Win g, float* __restrict__ h) {
    const int64_t n = (int64_t)C * H * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int xx = (int)(i % W);
        const int64_t row = i - xx;
        float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
        for (int k = 0; k < kWin; ++k) {
            const int q = xx + k - kRad;
            if (q < 0 || q >= W) continue;
            const float u = x[row + q], v = y[row + q], w = g.w[k];
            a = fmaf(w, u, a); b = fmaf(w, v, b);
            aa = fmaf(w, u * u, aa); bb = fmaf(w, v * v, bb); ab = fmaf(w, u * v, ab);
        }
        h[i] = a; h[n + i] = b; h[2 * n + i] = aa; h[3 * n + i] = bb; h[4 * n + i] = ab;
    }
}

// vertical blur -> SSIM map -> partial maps g[3][n]; sum of S into *ssim_sum
__global__ void ssim_v5(const float* __restrict__ h, int C, int H, int W, Win g,
                        float* __restrict__ gp, float* __restrict__ ssim_sum) {
    const int64_t n = (int64_t)C * H * W;
    const float inv_n = 1.0f / (float)n;
    float local = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int xx = (int)(i % W);
        const int yy = (int)((i / W) % H);
        const int64_t plane = i - (int64_t)yy * W - xx;
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < kWin; ++k) {
            const int q = yy + k - kRad;
            if (q < 0 || q >= H) continue;
            const int64_t j = plane + (int64_t)q * W + xx;
            const float w = g.w[k];
#pragma unroll
            for (int c = 0; c < 5; ++c) m[c] = fmaf(w, h[c * n + j], m[c]);
        }
        const float mx = m[0], my = m[1];
        const float sx = m[2] - mx * mx, sy = m[3] - my * my, sxy = m[4] - mx * my;
        const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = sx + sy + kC2;
        const float S = (A1 * A2) / (B1 * B2);
        local += S;
        const float sS = S * inv_n;
        gp[i] = sS * (2.f * my / A1 - 2.f * my / A2 - 2.f * mx / B1 + 2.f * mx / B2);
        gp[n + i] = -sS / B2;
        gp[2 * n + i] = 2.f * sS / A2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if (lane_id() == 0) atomicAdd(ssim_sum, local);
}

__global__ void ssim_h3(const float* __restrict__ gp, int C, int H, int W, Win g,
                        float* __restrict__ t) {
    const int64_t n = (int64_t)C * H * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int xx = (int)(i % W);
        const int64_t row = i - xx;
        float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
        for (int k = 0; k < kWin; ++k) {
            const int q = xx + k - kRad;
            if (q < 0 || q >= W) continue;
            const float w = g.w[k];
            a = fmaf(w, gp[row + q], a);
            b = fmaf(w, gp[n + row + q], b);
            c = fmaf(w, gp[2 * n + row + q], c);
        }
        t[i] = a; t[n + i] = b; t[2 * n + i] = c;
    }
}

// vertical blur of the partial maps -> dSSIM/dx; dimg = (1-lam) sign(x-y)/n - lam dSSIM/dx;
// also the L1 sum into *l1_sum
__global__ void ssim_v3(const float* __restrict__ t, const float* __restrict__ x,
                        const float* __restrict__ y, int C, int H, int W, Win g, float lam,
                        float* __restrict__ dimg, float* __restrict__ l1_sum) {
    const int64_t n = (int64_t)C * H * W;
    const float inv_n = 1.0f / (float)n;
    float local = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int xx = (int)(i % W);
        const int yy = (int)((i / W) % H);
        const int64_t plane = i - (int64_t)yy * W - xx;
        float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
        for (int k = 0; k < kWin; ++k) {
            const int q = yy + k - kRad;
            if (q < 0 || q >= H) continue;
            const int64_t j = plane + (int64_t)q * W + xx;
            const float w = g.w[k];
            a = fmaf(w, t[j], a);
            b = fmaf(w, t[n + j], b);
            c = fmaf(w, t[2 * n + j], c);
        }
        const float xi = x[i], yi = y[i];
        const float dssim = a + 2.f * xi * b + yi * c;
        const float d = xi - yi;
        local += fabsf(d);
        const float sgn = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
        dimg[i] = (1.f - lam) * sgn - lam * dssim;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if (lane_id() == 0) atomicAdd(l1_sum, local);
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
    return sizeof(float) * ((size_t)8 * C * H * W + 4) + 512;
}

extern "C" ogs_status ogs_loss_l1_ssim(const float* img, const float* target, int32_t C,
                                       int32_t H, int32_t W, float lambda, float* dimg,
                                       float* loss, void* scratch, size_t scratch_bytes,
                                       void* stream) {
    if (!img || !target || !dimg || !scratch || C <= 0 || H <= 0 || W <= 0) return OGS_ERR_ARG;
    if (!(lambda >= 0.f && lambda <= 1.f)) return OGS_ERR_ARG;
    if (scratch_bytes < ogs_loss_l1_ssim_scratch_bytes(C, H, W) || !aligned(scratch, 16))
        return OGS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)C * H * W;
    Carver cv(scratch);
    float* h = cv.take<float>(5 * n);
    float* gp = cv.take<float>(3 * n);
    float* sums = cv.take<float>(4);
    float* t = h;   // the 5 blurred maps are dead once the partial maps exist
    const Win g = make_window();
    if (cudaMemsetAsync(sums, 0, 4 * sizeof(float), st) != cudaSuccess) return OGS_ERR_CUDA;
    const int grid = stride_grid(n, 256, 8);
    ssim_h5<<<grid, 256, 0, st>>>(img, target, C, H, W, g, h);
    ssim_v5<<<grid, 256, 0, st>>>(h, C, H, W, g, gp, sums);
    ssim_h3<<<grid, 256, 0, st>>>(gp, C, H, W, g, t);
    ssim_v3<<<grid, 256, 0, st>>>(t, img, target, C, H, W, g, lambda, dimg, sums + 1);
    if (loss) combine_loss<<<1, 32, 0, st>>>(sums, n, lambda, loss);
    return launch_status();
}
