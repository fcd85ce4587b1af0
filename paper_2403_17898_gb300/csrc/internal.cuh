// Internal helpers shared by the sm_103a kernels of the renderer (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ogs.h"

namespace ogs {

constexpr int kTile = 16;
constexpr int kSmCount = 152;          // GB300: 2 dies x 76 SMs

// Camera in the form the kernels use (passed by value as a kernel parameter).
struct Cam {
    float R[9];
    float c[3];
    float fx, fy, cx, cy;
    int W, H;
    float znear, d_max, s;
    float limx, limy;   // 1.3 * tan(half fov)
    int gx, gy;         // tile grid
};

inline Cam make_cam(const ogs_camera& k) {
    Cam c;
    for (int i = 0; i < 9; ++i) c.R[i] = k.R[i];
    for (int i = 0; i < 3; ++i) c.c[i] = k.campos[i];
    c.fx = k.fx; c.fy = k.fy; c.cx = k.cx; c.cy = k.cy;
    c.W = k.width; c.H = k.height;
    c.znear = k.znear; c.d_max = k.d_max; c.s = k.s;
    c.limx = (float)(1.3 * (double)k.width / (2.0 * (double)k.fx));
    c.limy = (float)(1.3 * (double)k.height / (2.0 * (double)k.fy));
    c.gx = (k.width + kTile - 1) / kTile;
    c.gy = (k.height + kTile - 1) / kTile;
    return c;
}

inline bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

inline ogs_status launch_status() {
    return cudaGetLastError() == cudaSuccess ? OGS_OK : OGS_ERR_CUDA;
}

// Grid for a grid-stride kernel over up to `cap` items: enough blocks to cover the items,
// capped at `per_sm` resident blocks on every SM.
inline int stride_grid(int64_t cap, int block, int per_sm) {
    int64_t need = (cap + block - 1) / block;
    int64_t lim = (int64_t)kSmCount * per_sm;
    if (need < 1) need = 1;
    return (int)(need < lim ? need : lim);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Carve 256-byte-aligned sub-buffers out of a caller-provided scratch block.
struct Carver {
    char* base;
    size_t off = 0;
    __host__ explicit Carver(void* p) : base((char*)p) {}
    template <class T>
    __host__ T* take(size_t n) {
        off = (off + 255) & ~(size_t)255;
        T* p = (T*)(base ? base + off : nullptr);
        off += n * sizeof(T);
        return p;
    }
};

}  // namespace ogs
