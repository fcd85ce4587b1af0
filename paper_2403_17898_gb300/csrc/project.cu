// EWA projection of 3D Gaussians to screen-space Gaussians and their 16x16 tile extent
// (Sec. 3.1, Eq. 1: Sigma = R S S^T R^T, projected with the local affine Jacobian).
//
// One thread per Gaussian, grid-stride over the device-side count.  HBM-bound: reads 56 B of
// Gaussian SoA, writes a 48 B record, 4 B depth key, 8 B rect and 4 B tile count; optionally
// also counts the pairs of every tile (the first step of building the per-tile lists).
#include "internal.cuh"

namespace ogs {
namespace {

constexpr int kProjThreads = 256;

struct ProjArgs {
    ogs_gaussians g;
    const uint32_t* count;   // device count or null
    int64_t n_fixed;
    int rel;
    Cam cam;
    float4* rec;
    uint32_t* depth_key;
    uint2* rect;
    uint32_t* tiles;
    uint32_t* tile_count;    // optional per-tile pair counts (zeroed before the launch)
};

// Adds every lane's rectangle to the per-tile counts.  All 32 lanes call it.  The first tile
// of each lane is added with one atomic per distinct tile of the warp (the k Gaussians of an
// anchor sit in consecutive lanes and mostly share it); the rest of a small rectangle by its
// lane, and rectangles of more than kOwnTiles tiles by the whole warp.
constexpr uint32_t kOwnTiles = 8;

__device__ __forceinline__ void count_tiles(uint32_t* tc, int gx, uint2 rc, uint32_t ntiles) {
    const uint32_t x0 = rc.x & 0xFFFFu, y0 = rc.x >> 16, x1 = rc.y & 0xFFFFu;
    const uint32_t w = x1 - x0;
    const bool own = ntiles > 0 && ntiles <= kOwnTiles;
    const uint32_t t0 = own ? y0 * (uint32_t)gx + x0 : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xffffffffu, t0);
    if (own && lane_id() == (uint32_t)(__ffs(peers) - 1)) atomicAdd(tc + t0, (uint32_t)__popc(peers));
    if (own)
        for (uint32_t i = 1; i < ntiles; ++i) atomicAdd(tc + (y0 + i / w) * (uint32_t)gx + x0 + i % w, 1u);
    uint32_t big = __ballot_sync(0xffffffffu, ntiles > kOwnTiles);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const uint2 r = make_uint2(__shfl_sync(0xffffffffu, rc.x, src),
                                   __shfl_sync(0xffffffffu, rc.y, src));
        const uint32_t bx0 = r.x & 0xFFFFu, by0 = r.x >> 16, bw = (r.y & 0xFFFFu) - bx0;
        const uint32_t bn = bw * ((r.y >> 16) - by0);
        for (uint32_t i = lane_id(); i < bn; i += 32)
            atomicAdd(tc + (by0 + i / bw) * (uint32_t)gx + bx0 + i % bw, 1u);
    }
}

__global__ void __launch_bounds__(kProjThreads) project_kernel(ProjArgs a) {
    const Cam& c = a.cam;
    const int64_t n = a.count ? (int64_t)*a.count : a.n_fixed;
    // uniform trip count per warp, so the tile counting can use full-warp intrinsics
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gi = base + threadIdx.x;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
        uint32_t dkey = 0xFFFFFFFFu, ntiles = 0;
        uint2 rc = make_uint2(0, 0);
        const float o = gi < n ? a.g.opac[gi] : 0.0f;
        if (o > 0.0f) {
            float m0 = a.g.means[3 * gi], m1 = a.g.means[3 * gi + 1], m2 = a.g.means[3 * gi + 2];
            if (!a.rel) { m0 -= c.c[0]; m1 -= c.c[1]; m2 -= c.c[2]; }
            const float px = c.R[0] * m0 + c.R[1] * m1 + c.R[2] * m2;
            const float py = c.R[3] * m0 + c.R[4] * m1 + c.R[5] * m2;
            const float pz = c.R[6] * m0 + c.R[7] * m1 + c.R[8] * m2;
            if (pz > c.znear) {
                const float4 q = *reinterpret_cast<const float4*>(a.g.quats + 4 * gi);
                const float s0 = a.g.scales[3 * gi], s1 = a.g.scales[3 * gi + 1],
                            s2 = a.g.scales[3 * gi + 2];
                const float w = q.x, x = q.y, y = q.z, z = q.w;
                // M = R(q) S
                const float M00 = (1.f - 2.f * (y * y + z * z)) * s0, M01 = 2.f * (x * y - w * z) * s1,
                            M02 = 2.f * (x * z + w * y) * s2;
                const float M10 = 2.f * (x * y + w * z) * s0, M11 = (1.f - 2.f * (x * x + z * z)) * s1,
                            M12 = 2.f * (y * z - w * x) * s2;
                const float M20 = 2.f * (x * z - w * y) * s0, M21 = 2.f * (y * z + w * x) * s1,
                            M22 = (1.f - 2.f * (x * x + y * y)) * s2;
                // Sigma = M M^T (symmetric)
                const float S00 = M00 * M00 + M01 * M01 + M02 * M02;
                const float S01 = M00 * M10 + M01 * M11 + M02 * M12;
                const float S02 = M00 * M20 + M01 * M21 + M02 * M22;
                const float S11 = M10 * M10 + M11 * M11 + M12 * M12;
                const float S12 = M10 * M20 + M11 * M21 + M12 * M22;
                const float S22 = M20 * M20 + M21 * M21 + M22 * M22;
                // Jacobian of the perspective map at the (frustum-clamped) centre
                const float iz = 1.0f / pz;
                const float tx = fminf(fmaxf(px * iz, -c.limx), c.limx) * pz;
                const float ty = fminf(fmaxf(py * iz, -c.limy), c.limy) * pz;
                const float j00 = c.fx * iz, j02 = -c.fx * tx * iz * iz;
                const float j11 = c.fy * iz, j12 = -c.fy * ty * iz * iz;
                // T = J W (2x3)
                const float T00 = j00 * c.R[0] + j02 * c.R[6], T01 = j00 * c.R[1] + j02 * c.R[7],
                            T02 = j00 * c.R[2] + j02 * c.R[8];
                const float T10 = j11 * c.R[3] + j12 * c.R[6], T11 = j11 * c.R[4] + j12 * c.R[7],
                            T12 = j11 * c.R[5] + j12 * c.R[8];
                // cov2 = T Sigma T^T
                const float U0 = S00 * T00 + S01 * T01 + S02 * T02;
                const float U1 = S01 * T00 + S11 * T01 + S12 * T02;
                const float U2 = S02 * T00 + S12 * T01 + S22 * T02;
                const float V0 = S00 * T10 + S01 * T11 + S02 * T12;
                const float V1 = S01 * T10 + S11 * T11 + S12 * T12;
                const float V2 = S02 * T10 + S12 * T11 + S22 * T12;
                const float ca = T00 * U0 + T01 * U1 + T02 * U2 + 0.3f;
                const float cb = T10 * U0 + T11 * U1 + T12 * U2;
                const float cc = T10 * V0 + T11 * V1 + T12 * V2 + 0.3f;
                const float det = ca * cc - cb * cb;
                if (det > 0.0f) {
                    const float mid = 0.5f * (ca + cc);
                    const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
                    const float r = 3.0f * sqrtf(lam);
                    const float u = c.fx * px * iz + c.cx;
                    const float v = c.fy * py * iz + c.cy;
                    // tiles holding a pixel centre inside [u-r, u+r] x [v-r, v+r]
                    const float lo = -64.f, hix = 16.f * c.gx + 64.f, hiy = 16.f * c.gy + 64.f;
                    const float ex0 = fminf(fmaxf(ceilf(u - r), lo), hix);
                    const float ex1 = fminf(fmaxf(floorf(u + r), lo), hix);
                    const float ey0 = fminf(fmaxf(ceilf(v - r), lo), hiy);
                    const float ey1 = fminf(fmaxf(floorf(v + r), lo), hiy);
                    const int tx0 = max((int)floorf(ex0 * 0.0625f), 0);
                    const int tx1 = min((int)floorf(ex1 * 0.0625f) + 1, c.gx);
                    const int ty0 = max((int)floorf(ey0 * 0.0625f), 0);
                    const int ty1 = min((int)floorf(ey1 * 0.0625f) + 1, c.gy);
                    if (tx0 < tx1 && ty0 < ty1) {
                        const float id = 1.0f / det;
                        r0 = make_float4(u, v, cc * id, -cb * id);
                        r1 = make_float4(ca * id, o, a.g.colors[3 * gi], a.g.colors[3 * gi + 1]);
                        // alpha = o G < 1/255  <=>  power < -ln(255 o): the blend tests the
                        // exponent against this bound before evaluating exp
                        r2 = make_float4(a.g.colors[3 * gi + 2], pz, r, -logf(255.0f * o));
                        dkey = __float_as_uint(pz);
                        ntiles = (uint32_t)((tx1 - tx0) * (ty1 - ty0));
                        rc = make_uint2((uint32_t)tx0 | ((uint32_t)ty0 << 16),
                                        (uint32_t)tx1 | ((uint32_t)ty1 << 16));
                    }
                }
            }
        }
        if (gi < n) {
            a.rec[3 * gi] = r0;
            a.rec[3 * gi + 1] = r1;
            a.rec[3 * gi + 2] = r2;
            a.depth_key[gi] = dkey;
            a.rect[gi] = rc;
            a.tiles[gi] = ntiles;
        }
        if (a.tile_count) count_tiles(a.tile_count, c.gx, rc, ntiles);
    }
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" ogs_status ogs_project_bin(const ogs_gaussians* g, int64_t n_gauss, int32_t means_relative,
                                      const ogs_camera* cam, ogs_rec2d* rec, uint32_t* depth_key,
                                      uint32_t* rect, uint32_t* tiles, uint32_t* tile_count,
                                      ogs_counts* counts, void* stream) {
    if (!g || !cam || !rec || !depth_key || !rect || !tiles || n_gauss < 0) return OGS_ERR_ARG;
    if (!g->means || !g->scales || !g->quats || !g->opac || !g->colors) return OGS_ERR_ARG;
    if (!aligned(rec, 16) || !aligned(g->quats, 16) || !aligned(rect, 8)) return OGS_ERR_ARG;
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 16 * 65535 || cam->height > 16 * 65535)
        return OGS_ERR_ARG;
    const Cam cm = make_cam(*cam);
    cudaStream_t st = (cudaStream_t)stream;
    if (tile_count &&
        cudaMemsetAsync(tile_count, 0, sizeof(uint32_t) * (size_t)cm.gx * cm.gy, st) != cudaSuccess)
        return OGS_ERR_CUDA;
    if (n_gauss == 0) return OGS_OK;
    ProjArgs a{*g, counts ? &counts->n_gaussians : nullptr, n_gauss, means_relative, cm,
               reinterpret_cast<float4*>(rec), depth_key, reinterpret_cast<uint2*>(rect), tiles,
               tile_count};
    int grid = stride_grid(n_gauss, kProjThreads, 8);
    project_kernel<<<grid, kProjThreads, 0, st>>>(a);
    return launch_status();
}
