// EWA projection of 3D Gaussians to screen-space Gaussians and their 16x16 tile extent
// (Sec. 3.1, Eq. 1: Sigma = R S S^T R^T, projected with the local affine Jacobian).
//
// One thread per Gaussian, grid-stride over the device-side count.  HBM-bound: reads 56 B of
// Gaussian SoA, writes a 48 B record, 4 B depth key, 8 B rect and 4 B tile count; optionally
// also counts the pairs of every tile (the first step of building the per-tile lists).
#include "project_common.cuh"

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

__global__ void __launch_bounds__(kProjThreads) project_kernel(ProjArgs a) {
    const Cam& c = a.cam;
    const int64_t n = a.count ? (int64_t)*a.count : a.n_fixed;
    // uniform trip count per warp, so the tile counting can use full-warp intrinsics
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gi = base + threadIdx.x;
        ProjOut p;
        const float o = gi < n ? a.g.opac[gi] : 0.0f;
        if (o > 0.0f) {
            float m0 = a.g.means[3 * gi], m1 = a.g.means[3 * gi + 1], m2 = a.g.means[3 * gi + 2];
            if (!a.rel) { m0 -= c.c[0]; m1 -= c.c[1]; m2 -= c.c[2]; }
            p = project_one(c, m0, m1, m2, *reinterpret_cast<const float4*>(a.g.quats + 4 * gi),
                            a.g.scales[3 * gi], a.g.scales[3 * gi + 1], a.g.scales[3 * gi + 2],
                            o, a.g.colors[3 * gi], a.g.colors[3 * gi + 1],
                            a.g.colors[3 * gi + 2]);
        } else {
            p = project_one(c, 0.f, 0.f, 0.f, make_float4(1.f, 0.f, 0.f, 0.f), 0.f, 0.f, 0.f,
                            0.f, 0.f, 0.f, 0.f);    // culled: zero record
        }
        if (gi < n) {
            a.rec[3 * gi] = p.r0;
            a.rec[3 * gi + 1] = p.r1;
            a.rec[3 * gi + 2] = p.r2;
            a.depth_key[gi] = p.dkey;
            a.rect[gi] = p.rc;
            a.tiles[gi] = p.ntiles;
        }
        if (a.tile_count) count_tiles(a.tile_count, c.gx, p.rc, p.ntiles);
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
