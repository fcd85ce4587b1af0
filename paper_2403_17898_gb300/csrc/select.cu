// Anchor selection by octree level (Sec. 4.1.3, Eq. for L_hat) with the inference-time
// opacity blending of the next level, followed by an order-preserving compaction.
//
// HBM-bound streaming pass over the anchor SoA (pos 12 B + level 1 B + dL 4 B per anchor),
// read once: a single-pass order-preserving compaction.  Each CTA stages one tile of anchors
// in shared memory with TMA bulk copies (so the whole tile's bytes are in flight at once),
// evaluates the predicate from there, ranks its kept anchors with warp ballots, obtains the
// tile's output offset by a decoupled look-back over the predecessor tiles' published counts
// (tiles are taken in ticket order, so every predecessor is already running) and scatters,
// so sel_idx stays in ascending anchor order without a second pass or a global sort.
#include "internal.cuh"
#include "tc.cuh"

namespace ogs {
namespace {

constexpr int kSelThreads = 256;
constexpr int kSelItems = 8;
constexpr int kSelWarps = kSelThreads / 32;
constexpr int kSelChunk = kSelThreads * kSelItems;   // anchors per tile (one CTA)
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

// Returns true if an anchor at (px, py, pz) with level `lvl` and LOD bias `dl` is kept; w
// receives its opacity weight.
__device__ __forceinline__ bool keep_anchor(const SelArgs& a, float px, float py, float pz,
                                           uint32_t lvl, float dl, float& w) {
    const Cam& c = a.cam;
    float dx = px - c.c[0];
    float dy = py - c.c[1];
    float dz = pz - c.c[2];
    // visibility of the anchor centre: in front of the near plane, within 1.3x half-fov
    float zc = c.R[6] * dx + c.R[7] * dy + c.R[8] * dz;
    float xc = c.R[0] * dx + c.R[1] * dy + c.R[2] * dz;
    float yc = c.R[3] * dx + c.R[4] * dy + c.R[5] * dz;
    if (!(zc > c.znear) || fabsf(xc) > c.limx * zc || fabsf(yc) > c.limy * zc) return false;
    // fractional level from the viewing distance plus the anchor's LOD bias, clamped
    float d = sqrtf(dx * dx + dy * dy + dz * dz);
    float Lraw = log2f(c.d_max / (d * c.s)) + dl;
    float Ls = fminf(fmaxf(Lraw, 0.0f), (float)(a.NL - 1));
    float Lh = floorf(Ls);
    float L = (float)lvl;
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

// Single pass: each CTA takes the next tile by ticket, evaluates the predicate for its
// kSelChunk anchors (coalesced), counts them per (item, warp), publishes its count, looks
// back for its exclusive offset and scatters its kept anchors in ascending order.
__global__ void __launch_bounds__(kSelThreads) select_onepass(SelArgs a,
                                                              unsigned long long* status,
                                                              uint32_t* ticket, int nb,
                                                              uint32_t* sel_idx, float* sel_w,
                                                              int64_t cap, ogs_counts* counts,
                                                              int bulk) {
    __shared__ __align__(16) float s_pos[3 * kSelChunk];
    __shared__ __align__(16) float s_dl[kSelChunk];
    __shared__ __align__(16) uint8_t s_lvl[kSelChunk];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_cnt[kSelItems * kSelWarps];
    __shared__ uint32_t s_agg;
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * kSelChunk;
    const int n_here = (int)min((int64_t)kSelChunk, a.N - base);
    const unsigned warp = threadIdx.x >> 5;
    // stage the tile's anchor SoA in shared memory: three TMA bulk copies for a full tile of
    // aligned arrays, cooperative loads otherwise
    if (bulk && n_here == kSelChunk) {
        if (threadIdx.x == 0) {
            tc::mbar_init(&mbar, 1);
            tc::mbar_expect_tx(&mbar, (3 * 4 + 4 + 1) * kSelChunk);
            tc::bulk_load(s_pos, a.pos + 3 * base, 3 * 4 * kSelChunk, &mbar);
            tc::bulk_load(s_dl, a.dL + base, 4 * kSelChunk, &mbar);
            tc::bulk_load(s_lvl, a.level + base, kSelChunk, &mbar);
        }
        __syncthreads();                              // barrier initialised before anyone polls
        if (!tc::mbar_wait(&mbar, 0, kSpinLimit)) {
            atomicExch(&counts->timeout, 1u);
            tc::mbar_wait(&mbar, 0, kSpinLimit);      // copies may still be landing
        }
    } else {
        for (int e = threadIdx.x; e < 3 * n_here; e += kSelThreads) s_pos[e] = a.pos[3 * base + e];
        for (int e = threadIdx.x; e < n_here; e += kSelThreads) {
            s_dl[e] = a.dL[base + e];
            s_lvl[e] = a.level[base + e];
        }
        __syncthreads();
    }
    uint32_t keepbits = 0;
    float w[kSelItems];
    unsigned bal[kSelItems];
#pragma unroll
    for (int it = 0; it < kSelItems; ++it) {
        const int l = it * kSelThreads + threadIdx.x;
        w[it] = 0.0f;
        const bool keep = l < n_here && keep_anchor(a, s_pos[3 * l], s_pos[3 * l + 1],
                                                    s_pos[3 * l + 2], s_lvl[l], s_dl[l], w[it]);
        keepbits |= (uint32_t)keep << it;
        bal[it] = __ballot_sync(0xffffffffu, keep);
        if (lane_id() == 0) s_cnt[it * kSelWarps + warp] = __popc(bal[it]);
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive scan of the 64 (item, warp) counts in output order, two per lane
        const uint32_t c0 = s_cnt[2 * lane_id()], c1 = s_cnt[2 * lane_id() + 1];
        uint32_t x = c0 + c1;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (unsigned)o) x += y;
        }
        __syncwarp();
        s_cnt[2 * lane_id()] = x - c0 - c1;
        s_cnt[2 * lane_id() + 1] = x - c1;
        if (lane_id() == 31) s_agg = x;
    }
    __syncthreads();
    const unsigned long long agg = s_agg;
    const unsigned long long excl0 =
        block_tile_offset<kSelThreads>(status, tile, agg, &counts->timeout);
    if (threadIdx.x == 0 && tile == (uint32_t)nb - 1) {      // the last tile knows the total
        const unsigned long long total = excl0 + agg;
        const uint32_t m = total > (unsigned long long)cap ? (uint32_t)cap : (uint32_t)total;
        counts->n_selected = m;
        counts->n_gaussians = m * (uint32_t)a.k;
        counts->need_selected = total > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)total;
        if (total > (unsigned long long)cap) atomicOr(&counts->overflow, 1u);
    }
    const unsigned long long excl = excl0;
#pragma unroll
    for (int it = 0; it < kSelItems; ++it) {
        if ((keepbits >> it) & 1u) {
            const unsigned long long p = excl + s_cnt[it * kSelWarps + warp] +
                                         __popc(bal[it] & lanemask_lt());
            if (p < (unsigned long long)cap) {
                sel_idx[p] = (uint32_t)(base + it * kSelThreads + threadIdx.x);
                sel_w[p] = w[it];
            }
        }
    }
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" size_t ogs_lod_select_scratch_bytes(int64_t N) {
    int64_t nb = (N + kSelChunk - 1) / kSelChunk;
    return (size_t)((nb < 1 ? 1 : nb) + 1) * sizeof(unsigned long long) + 256;
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
    // tile status words, then the ticket counter: all zero before the pass
    unsigned long long* status = (unsigned long long*)scratch;
    uint32_t* ticket = (uint32_t*)(status + nb);
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (nb + 1), st) != cudaSuccess)
        return OGS_ERR_CUDA;
    const int bulk = aligned(pos, 16) && aligned(dL, 16) && aligned(level, 16);
    select_onepass<<<nb, kSelThreads, 0, st>>>(a, status, ticket, nb, sel_idx, sel_w, sel_cap,
                                               counts, bulk);
    return launch_status();
}

extern "C" const char* ogs_version(void) { return "ogs-gb300 0.1 (sm_103a)"; }
