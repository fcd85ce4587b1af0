// Anchor selection by octree level (Sec. 4.1.3, Eq. for L_hat) with the inference-time
// opacity blending of the next level, followed by an order-preserving compaction.
//
// HBM-bound streaming pass over the anchor SoA (pos 12 B + level 1 B + dL 4 B per anchor).
// Compaction is count -> scan of block counts -> scatter: the scatter pass re-evaluates the
// predicate (cheaper than storing per-anchor flags) and ranks kept anchors with warp ballots,
// so sel_idx stays in ascending anchor order without a global sort.
#include "internal.cuh"

namespace ogs {
namespace {

constexpr int kSelThreads = 256;
constexpr int kSelItems = 4;
constexpr int kSelChunk = kSelThreads * kSelItems;   // anchors per block

struct SelArgs {
    const float* pos;
    const uint8_t* level;
    const float* dL;
    int64_t N;
    int NL;
    int k;
    int infer;
    Cam cam;
};

// Returns true if anchor j is kept; w receives its opacity weight.
__device__ __forceinline__ bool keep_anchor(const SelArgs& a, int64_t j, float& w) {
    const Cam& c = a.cam;
    float dx = a.pos[3 * j] - c.c[0];
    float dy = a.pos[3 * j + 1] - c.c[1];
    float dz = a.pos[3 * j + 2] - c.c[2];
    // visibility of the anchor centre: in front of the near plane, within 1.3x half-fov
    float zc = c.R[6] * dx + c.R[7] * dy + c.R[8] * dz;
    float xc = c.R[0] * dx + c.R[1] * dy + c.R[2] * dz;
    float yc = c.R[3] * dx + c.R[4] * dy + c.R[5] * dz;
    if (!(zc > c.znear) || fabsf(xc) > c.limx * zc || fabsf(yc) > c.limy * zc) return false;
    // fractional level from the viewing distance plus the anchor's LOD bias, clamped
    float d = sqrtf(dx * dx + dy * dy + dz * dz);
    float Lraw = log2f(c.d_max / (d * c.s)) + a.dL[j];
    float Ls = fminf(fmaxf(Lraw, 0.0f), (float)(a.NL - 1));
    float Lh = floorf(Ls);
    float L = (float)a.level[j];
    if (L <= Lh) {
        w = 1.0f;
        return true;
    }
    if (a.infer && L == Lh + 1.0f && Ls > Lh) {
        w = Ls - Lh;
        return true;
    }
    return false;
}

__global__ void __launch_bounds__(kSelThreads) select_count(SelArgs a, uint32_t* block_count) {
    __shared__ uint32_t warp_tot[kSelThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kSelChunk;
    uint32_t mine = 0;
#pragma unroll 4
    for (int it = 0; it < kSelItems; ++it) {
        int64_t j = base + it * kSelThreads + threadIdx.x;
        float w;
        bool keep = j < a.N && keep_anchor(a, j, w);
        mine += __popc(__ballot_sync(0xffffffffu, keep));
    }
    if (lane_id() == 0) warp_tot[threadIdx.x >> 5] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int i = 0; i < kSelThreads / 32; ++i) s += warp_tot[i];
        block_count[blockIdx.x] = s;
    }
}

// Exclusive scan of per-block counts by one block; publishes M and the overflow state.
__global__ void __launch_bounds__(1024) select_scan(uint32_t* block_count, int nb, int64_t cap,
                                                     int k, ogs_counts* counts) {
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        int b = b0 + threadIdx.x;
        uint32_t v = b < nb ? block_count[b] : 0;
        // inclusive warp scan
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (unsigned)o) x += y;
        }
        if (lane_id() == 31) warp_sum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t s = warp_sum[threadIdx.x];
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane_id() >= (unsigned)o) s += y;
            }
            warp_sum[threadIdx.x] = s;   // inclusive over warps
        }
        __syncthreads();
        uint32_t wpre = (threadIdx.x >> 5) ? warp_sum[(threadIdx.x >> 5) - 1] : 0;
        uint32_t excl = carry + wpre + x - v;
        if (b < nb) block_count[b] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        uint32_t total = carry;
        uint32_t m = total > (uint64_t)cap ? (uint32_t)cap : total;
        counts->n_selected = m;
        counts->n_gaussians = m * (uint32_t)k;
        counts->need_selected = total;
        if (total > (uint64_t)cap) atomicOr(&counts->overflow, 1u);
    }
}

__global__ void __launch_bounds__(kSelThreads) select_scatter(SelArgs a, const uint32_t* block_off,
                                                              uint32_t* sel_idx, float* sel_w,
                                                              int64_t cap) {
    __shared__ uint32_t warp_cnt[kSelThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kSelChunk;
    const unsigned warp = threadIdx.x >> 5;
    uint32_t running = block_off[blockIdx.x];
    for (int it = 0; it < kSelItems; ++it) {
        int64_t j = base + it * kSelThreads + threadIdx.x;
        float w = 0.0f;
        bool keep = j < a.N && keep_anchor(a, j, w);
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane_id() == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        uint32_t wpre = 0, tot = 0;
#pragma unroll
        for (int i = 0; i < kSelThreads / 32; ++i) {
            uint32_t c = warp_cnt[i];
            wpre += (i < (int)warp) ? c : 0;
            tot += c;
        }
        if (keep) {
            uint64_t p = (uint64_t)running + wpre + __popc(bal & lanemask_lt());
            if (p < (uint64_t)cap) {
                sel_idx[p] = (uint32_t)j;
                sel_w[p] = w;
            }
        }
        running += tot;
        __syncthreads();
    }
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" size_t ogs_lod_select_scratch_bytes(int64_t N) {
    int64_t nb = (N + kSelChunk - 1) / kSelChunk;
    return (size_t)(nb < 1 ? 1 : nb) * sizeof(uint32_t) + 256;
}

extern "C" ogs_status ogs_lod_select(const float* pos, const uint8_t* level, const float* dL,
                                     int64_t N, int32_t NL, int32_t k, const ogs_camera* cam,
                                     int32_t infer, uint32_t* sel_idx, float* sel_w,
                                     int64_t sel_cap, ogs_counts* counts, void* scratch,
                                     size_t scratch_bytes, void* stream) {
    if (!pos || !level || !dL || !cam || !sel_idx || !sel_w || !counts || !scratch)
        return OGS_ERR_ARG;
    if (N < 0 || N > 0xFFFFFFFFll || NL < 1 || NL > 255 || k < 1 || sel_cap < 0)
        return OGS_ERR_ARG;
    if (cam->width <= 0 || cam->height <= 0 || !(cam->d_max > 0) || !(cam->s > 0))
        return OGS_ERR_ARG;
    if (scratch_bytes < ogs_lod_select_scratch_bytes(N) || !aligned(scratch, 16)) return OGS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    SelArgs a{pos, level, dL, N, NL, k, infer, make_cam(*cam)};
    int nb = (int)((N + kSelChunk - 1) / kSelChunk);
    if (nb < 1) nb = 1;
    uint32_t* block = (uint32_t*)scratch;
    select_count<<<nb, kSelThreads, 0, st>>>(a, block);
    select_scan<<<1, 1024, 0, st>>>(block, nb, sel_cap, k, counts);
    select_scatter<<<nb, kSelThreads, 0, st>>>(a, block, sel_idx, sel_w, sel_cap);
    return launch_status();
}

extern "C" const char* ogs_version(void) { return "ogs-gb300 0.1 (sm_103a)"; }
