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

// Appearance codes (Sec. 4.4): at most this many values per anchor, so that a code fits the
// zero-padded K columns 40..47 of the tensor-core decoders' first layer.
constexpr int kMaxApp = 8;

// The appearance fields of a decoder are usable: A in [0, kMaxApp], both arrays given if A > 0.
inline bool app_ok(const ogs_mlp& m) {
    return m.A >= 0 && m.A <= kMaxApp && (m.A == 0 || (m.w1_app && m.app));
}

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

// Programmatic dependent launch along the frame's kernel chain: a kernel launched with
// launch_pdl may be scheduled while its predecessor in the stream is still running; it calls
// pdl_wait() before touching any memory the earlier work writes (the wait returns once the
// predecessor grid has completed and its writes are visible), then pdl_trigger() so that its
// own successor can be scheduled early in turn.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
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


// ---------------------------------------------------------------------------------------
// Single-pass order-preserving compaction: tiles taken in ticket order publish their count
// in a status word (flag in the top two bits) and find their output offset by a decoupled
// look-back over their predecessors.
// ---------------------------------------------------------------------------------------
constexpr uint32_t kSpinLimit = 1u << 20;                  // polls of one status word
constexpr unsigned long long kFlagAgg = 1ull << 62;        // tile's own count published
constexpr unsigned long long kFlagPrefix = 2ull << 62;     // inclusive prefix published
constexpr unsigned long long kValMask = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long load_status(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void store_status(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

// Exclusive output offset of tile `tile` (count `agg`) by a decoupled look-back, called by
// every thread of the CTA: each round inspects the kThreads nearest unresolved predecessors
// at once (one status word per thread), adds their counts up to the nearest one that has
// published an inclusive prefix, and stops there; a thread stops waiting for its own
// predecessor as soon as a nearer one is known to hold a prefix.  All tiles of a launch run at about the
// same time, so a wide window keeps the chain of rounds short.  Predecessors hold earlier
// tickets, so they are running or done and publish without waiting on this tile; every wait
// is still bounded: on expiry the prefix is published anyway (so successors finish) and
// *timeout is set, which marks the whole result invalid.
template <int kThreads>
__device__ __forceinline__ unsigned long long block_tile_offset(unsigned long long* status,
                                                                uint32_t tile,
                                                                unsigned long long agg,
                                                                uint32_t* timeout) {
    __shared__ unsigned long long s_sum[kThreads / 32];
    __shared__ int s_stop;
    __shared__ int s_bad;
    if (tile == 0) {
        if (threadIdx.x == 0) store_status(status, kFlagPrefix | agg);
        return 0;
    }
    if (threadIdx.x == 0) store_status(status + tile, kFlagAgg | agg);
    unsigned long long excl = 0;
    bool ok = true;
    for (int64_t end = tile; end > 0; end -= kThreads) {
        const int64_t idx = end - 1 - (int64_t)threadIdx.x;
        if (threadIdx.x == 0) { s_stop = kThreads; s_bad = 0; }
        __syncthreads();
        unsigned long long v = kFlagPrefix;             // before tile 0: prefix 0
        if (idx >= 0) {
            uint32_t polls = 0;
            for (;;) {
                v = load_status(status + idx);
                const uint32_t f = (uint32_t)(v >> 62);
                if (f == 2) { atomicMin(&s_stop, (int)threadIdx.x); break; }
                if (f == 1) break;
                // a nearer predecessor already holds a prefix: this one is not needed
                if (*(volatile int*)&s_stop < (int)threadIdx.x) break;
                if (++polls > kSpinLimit) break;
                __nanosleep(32);
            }
        } else {
            atomicMin(&s_stop, (int)threadIdx.x);
        }
        __syncthreads();
        const int stop = s_stop;                         // nearest prefix in this window
        const bool mine = (int)threadIdx.x <= stop;
        if (mine && (v >> 62) == 0) s_bad = 1;
        unsigned long long add = mine ? (v & kValMask) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) add += __shfl_xor_sync(0xffffffffu, add, o);
        if (lane_id() == 0) s_sum[threadIdx.x >> 5] = add;
        __syncthreads();
        if (s_bad) { ok = false; break; }
        unsigned long long round = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) round += s_sum[w];
        excl += round;
        __syncthreads();                                 // s_sum, s_stop reused next round
        if (stop < kThreads) break;
    }
    if (threadIdx.x == 0) {
        store_status(status + tile, kFlagPrefix | ((excl + agg) & kValMask));
        if (!ok) atomicExch(timeout, 1u);
    }
    return excl;
}

}  // namespace ogs
