// EWA projection of one 3D Gaussian to its screen-space record and 16x16 tile extent (Sec. 3.1,
// Eq. 1: Sigma = R S S^T R^T, projected with the local affine Jacobian), and the per-tile pair
// counting.  Shared by ogs_project_bin and the fused decode + projection, so both produce the
// same bits.
#pragma once

#include "internal.cuh"

namespace ogs {

struct ProjOut {
    float4 r0, r1, r2;   // the 48-byte record (zeros when the Gaussian is culled)
    uint32_t dkey;       // depth key (float bits of the camera-space depth), ~0 when culled
    uint32_t ntiles;     // tiles of its rectangle (0 when culled)
    uint2 rc;            // (x0 | y0 << 16, x1 | y1 << 16): tiles [x0, x1) x [y0, y1)
};

// Every product and sum below is an explicit round-to-nearest intrinsic, so the compiler cannot
// contract them differently in the kernels that inline this function.
__device__ __forceinline__ float pm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float pa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float pf(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// a0 b0 + a1 b1 + a2 b2
__device__ __forceinline__ float dot3(float a0, float a1, float a2, float b0, float b1, float b2) {
    return pf(a2, b2, pf(a1, b1, pm(a0, b0)));
}

// m: camera-relative mean (world axes); q = (w, x, y, z) unit quaternion; s: scales; o: opacity
// (culled when o <= 0); col: colour.
__device__ __forceinline__ ProjOut project_one(const Cam& c, float m0, float m1, float m2,
                                               float4 q, float s0, float s1, float s2, float o,
                                               float col0, float col1, float col2) {
    ProjOut out;
    out.r0 = make_float4(0.f, 0.f, 0.f, 0.f);
    out.r1 = out.r0;
    out.r2 = out.r0;
    out.dkey = 0xFFFFFFFFu;
    out.ntiles = 0;
    out.rc = make_uint2(0, 0);
    if (!(o > 0.0f)) return out;
    const float px = dot3(c.R[0], c.R[1], c.R[2], m0, m1, m2);
    const float py = dot3(c.R[3], c.R[4], c.R[5], m0, m1, m2);
    const float pz = dot3(c.R[6], c.R[7], c.R[8], m0, m1, m2);
    if (!(pz > c.znear)) return out;
    const float w = q.x, x = q.y, y = q.z, z = q.w;
    const float xx = pm(x, x), yy = pm(y, y), zz = pm(z, z);
    const float xy = pm(x, y), xz = pm(x, z), yz = pm(y, z);
    const float wx = pm(w, x), wy = pm(w, y), wz = pm(w, z);
    // M = R(q) S
    const float M00 = pm(pf(-2.f, pa(yy, zz), 1.f), s0), M01 = pm(pm(2.f, pa(xy, -wz)), s1),
                M02 = pm(pm(2.f, pa(xz, wy)), s2);
    const float M10 = pm(pm(2.f, pa(xy, wz)), s0), M11 = pm(pf(-2.f, pa(xx, zz), 1.f), s1),
                M12 = pm(pm(2.f, pa(yz, -wx)), s2);
    const float M20 = pm(pm(2.f, pa(xz, -wy)), s0), M21 = pm(pm(2.f, pa(yz, wx)), s1),
                M22 = pm(pf(-2.f, pa(xx, yy), 1.f), s2);
    // Sigma = M M^T (symmetric)
    const float S00 = dot3(M00, M01, M02, M00, M01, M02);
    const float S01 = dot3(M00, M01, M02, M10, M11, M12);
    const float S02 = dot3(M00, M01, M02, M20, M21, M22);
    const float S11 = dot3(M10, M11, M12, M10, M11, M12);
    const float S12 = dot3(M10, M11, M12, M20, M21, M22);
    const float S22 = dot3(M20, M21, M22, M20, M21, M22);
    // Jacobian of the perspective map at the (frustum-clamped) centre
    const float iz = __frcp_rn(pz);
    const float tx = pm(fminf(fmaxf(pm(px, iz), -c.limx), c.limx), pz);
    const float ty = pm(fminf(fmaxf(pm(py, iz), -c.limy), c.limy), pz);
    const float iz2 = pm(iz, iz);
    const float j00 = pm(c.fx, iz), j02 = -pm(pm(c.fx, tx), iz2);
    const float j11 = pm(c.fy, iz), j12 = -pm(pm(c.fy, ty), iz2);
    // T = J W (2x3)
    const float T00 = pf(j02, c.R[6], pm(j00, c.R[0])), T01 = pf(j02, c.R[7], pm(j00, c.R[1])),
                T02 = pf(j02, c.R[8], pm(j00, c.R[2]));
    const float T10 = pf(j12, c.R[6], pm(j11, c.R[3])), T11 = pf(j12, c.R[7], pm(j11, c.R[4])),
                T12 = pf(j12, c.R[8], pm(j11, c.R[5]));
    // cov2 = T Sigma T^T
    const float U0 = dot3(S00, S01, S02, T00, T01, T02);
    const float U1 = dot3(S01, S11, S12, T00, T01, T02);
    const float U2 = dot3(S02, S12, S22, T00, T01, T02);
    const float V0 = dot3(S00, S01, S02, T10, T11, T12);
    const float V1 = dot3(S01, S11, S12, T10, T11, T12);
    const float V2 = dot3(S02, S12, S22, T10, T11, T12);
    const float ca = pa(dot3(T00, T01, T02, U0, U1, U2), 0.3f);
    const float cb = dot3(T10, T11, T12, U0, U1, U2);
    const float cc = pa(dot3(T10, T11, T12, V0, V1, V2), 0.3f);
    const float det = pf(ca, cc, -pm(cb, cb));
    if (!(det > 0.0f)) return out;
    const float mid = pm(0.5f, pa(ca, cc));
    const float lam = pa(mid, __fsqrt_rn(fmaxf(0.1f, pf(mid, mid, -det))));
    const float r = pm(3.0f, __fsqrt_rn(lam));
    const float u = pf(pm(c.fx, px), iz, c.cx);
    const float v = pf(pm(c.fy, py), iz, c.cy);
    // tiles holding a pixel centre inside [u-r, u+r] x [v-r, v+r]
    const float lo = -64.f, hix = 16.f * c.gx + 64.f, hiy = 16.f * c.gy + 64.f;
    const float ex0 = fminf(fmaxf(ceilf(pa(u, -r)), lo), hix);
    const float ex1 = fminf(fmaxf(floorf(pa(u, r)), lo), hix);
    const float ey0 = fminf(fmaxf(ceilf(pa(v, -r)), lo), hiy);
    const float ey1 = fminf(fmaxf(floorf(pa(v, r)), lo), hiy);
    const int tx0 = max((int)floorf(ex0 * 0.0625f), 0);
    const int tx1 = min((int)floorf(ex1 * 0.0625f) + 1, c.gx);
    const int ty0 = max((int)floorf(ey0 * 0.0625f), 0);
    const int ty1 = min((int)floorf(ey1 * 0.0625f) + 1, c.gy);
    if (!(tx0 < tx1 && ty0 < ty1)) return out;
    const float id = __frcp_rn(det);
    out.r0 = make_float4(u, v, pm(cc, id), -pm(cb, id));
    out.r1 = make_float4(pm(ca, id), o, col0, col1);
    // alpha = o G < 1/255  <=>  power < -ln(255 o): the blend tests the exponent against this
    // bound before evaluating exp
    out.r2 = make_float4(col2, pz, r, -logf(pm(255.0f, o)));
    out.dkey = __float_as_uint(pz);
    out.ntiles = (uint32_t)((tx1 - tx0) * (ty1 - ty0));
    out.rc = make_uint2((uint32_t)tx0 | ((uint32_t)ty0 << 16), (uint32_t)tx1 | ((uint32_t)ty1 << 16));
    return out;
}

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

// Rectangles of more than kOwnTiles tiles go through the whole warp in chunks of kChunkTiles
// tiles.  bin_tiles hands each chunk to a list of deferred (Gaussian, chunk) entries that a
// second pass spreads over the whole grid, so that a warp holding many large near-camera
// Gaussians does not walk all their tiles alone; chunks that find the list full stay with
// the warp.
constexpr uint32_t kChunkTiles = 1024;

// Places tiles [lo, hi) of rectangle r (row-major inside it) for Gaussian g with key k: every
// lane of the warp takes one tile in 32, kFly atomics in flight before the stores.  All 32
// lanes call it with the same arguments.
template <uint32_t kFly>
__device__ __forceinline__ void bin_rect_range(uint32_t* tc, int gx, uint2 r, uint32_t lo,
                                               uint32_t hi, uint32_t g, uint32_t k,
                                               uint32_t cap, uint32_t* __restrict__ pair_key,
                                               uint32_t* __restrict__ pair_gauss) {
    const uint32_t bx0 = r.x & 0xFFFFu, by0 = r.x >> 16, bw = (r.y & 0xFFFFu) - bx0;
    for (uint32_t i0 = lo; i0 < hi; i0 += 32 * kFly) {
        uint32_t tt[kFly], sl[kFly];
#pragma unroll
        for (uint32_t j = 0; j < kFly; ++j) {
            const uint32_t i = i0 + j * 32 + lane_id();
            if (i < hi) {
                tt[j] = (by0 + i / bw) * (uint32_t)gx + bx0 + i % bw;
                sl[j] = atomicAdd(tc + tt[j], 1u);
            }
        }
#pragma unroll
        for (uint32_t j = 0; j < kFly; ++j) {
            const uint32_t i = i0 + j * 32 + lane_id();
            if (i < hi && sl[j] < cap) {
                const size_t o = (size_t)tt[j] * cap + sl[j];
                pair_gauss[o] = g;
                pair_key[o] = k;
            }
        }
    }
}

// count_tiles, and each pair placed at once: the atomic that counts a (Gaussian, tile) pair
// returns its slot in the tile's region of cap entries, where the Gaussian's id and depth key
// go (pair_gauss[t * cap + slot], pair_key[...]); slots at or past cap are counted, not
// written (the caller sees the overflow in the counts).  g and dkey are the lane's Gaussian.
// A lane issues all its atomics (up to kOwnTiles at a time) before the first store that needs
// a slot, so their round trips overlap instead of adding up.  A larger rectangle is cut into
// chunks of kChunkTiles tiles, appended as (g, chunk) to `defer` (defer_cap entries, the
// 64-bit counter n_defer counts every chunk offered); chunks past defer_cap are placed here.
__device__ __forceinline__ void bin_tiles(uint32_t* tc, int gx, uint2 rc, uint32_t ntiles,
                                          uint32_t g, uint32_t dkey, uint32_t cap,
                                          uint32_t* __restrict__ pair_key,
                                          uint32_t* __restrict__ pair_gauss,
                                          uint2* __restrict__ defer,
                                          unsigned long long* n_defer, uint32_t defer_cap) {
    const uint32_t x0 = rc.x & 0xFFFFu, y0 = rc.x >> 16, x1 = rc.y & 0xFFFFu;
    const uint32_t w = x1 - x0;
    const uint32_t lane = lane_id();
    // large rectangles first (their list state is dead before the small ones' slots are live)
    const bool is_big = ntiles > kOwnTiles;
    if (__any_sync(0xffffffffu, is_big)) {
        // chunks of the lane's rectangle, numbered across the warp by an inclusive scan
        const uint32_t bn = is_big ? w * ((rc.y >> 16) - y0) : 0;
        const uint32_t nch = (bn + kChunkTiles - 1) / kChunkTiles;
        uint32_t incl = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane >= o) incl += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(n_defer, (unsigned long long)total);
        first = __shfl_sync(0xffffffffu, first, 0);
        const unsigned long long mine = first + (incl - nch);    // this lane's first entry
        uint32_t kept = 0;                                       // chunks the list took
        if (mine < (unsigned long long)defer_cap) {
            const unsigned long long room = (unsigned long long)defer_cap - mine;
            kept = room < nch ? (uint32_t)room : nch;
        }
        for (uint32_t c = 0; c < kept; ++c) defer[mine + c] = make_uint2(g, c);
        // what the list could not take stays with the warp, one rectangle at a time (four
        // atomics in flight per lane: this path is rare and keeps the kernel's registers low)
        const uint32_t lo = kept * kChunkTiles;
        uint32_t left = __ballot_sync(0xffffffffu, lo < bn);
        while (left) {
            const int src = __ffs(left) - 1;
            left &= left - 1;
            const uint2 r = make_uint2(__shfl_sync(0xffffffffu, rc.x, src),
                                       __shfl_sync(0xffffffffu, rc.y, src));
            bin_rect_range<4>(tc, gx, r, __shfl_sync(0xffffffffu, lo, src),
                           __shfl_sync(0xffffffffu, bn, src), __shfl_sync(0xffffffffu, g, src),
                           __shfl_sync(0xffffffffu, dkey, src), cap, pair_key, pair_gauss);
        }
    }
    auto put = [&](uint32_t t, uint32_t slot) {
        if (slot < cap) {
            const size_t o = (size_t)t * cap + slot;
            pair_gauss[o] = g;
            pair_key[o] = dkey;
        }
    };
    const bool own = ntiles > 0 && ntiles <= kOwnTiles;
    const uint32_t t0 = own ? y0 * (uint32_t)gx + x0 : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xffffffffu, t0);
    const uint32_t leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (own && lane == leader) base = atomicAdd(tc + t0, (uint32_t)__popc(peers));
    if (own) {
        uint32_t tt[kOwnTiles], sl[kOwnTiles];
        uint32_t kx = 0, t = t0;                    // walks the rectangle row by row
#pragma unroll
        for (uint32_t i = 1; i < kOwnTiles; ++i) {
            if (++kx == w) {
                kx = 0;
                t += (uint32_t)gx - w + 1;
            } else {
                ++t;
            }
            tt[i] = t;
            if (i < ntiles) sl[i] = atomicAdd(tc + t, 1u);
        }
#pragma unroll
        for (uint32_t i = 1; i < kOwnTiles; ++i)
            if (i < ntiles) put(tt[i], sl[i]);
    }
    base = __shfl_sync(0xffffffffu, base, leader);
    if (own) put(t0, base + __popc(peers & lanemask_lt()));
}

}  // namespace ogs
