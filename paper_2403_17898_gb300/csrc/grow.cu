// Anchor growing and the LOD-bias update (Sec. 4.2.1).
//
//   ogs_grow_accumulate   per view: each visible Gaussian adds the norm of its view-space mean
//                         gradient (normalised device units) to its (anchor, slot) statistic
//   ogs_update_lod_bias   dL += eps for anchors whose average gradient exceeds 0.25 tau[L]
//   ogs_grow_anchors      next-level growing: every Gaussian whose average gradient passes
//                         tau[L] (or tau[L + 1]) proposes the voxel holding it, at level L
//                         (or L + 1); free voxels become new anchors, first proposal wins
//
// Growing runs on a voxel hash table (open addressing, linear probing, 64-bit keys packing
// the level and three 20-bit voxel coordinates; at most half full, so probes stay short):
//   1. clear the table;
//   2. one thread per existing anchor inserts its own voxel key with value 0;
//   3. one thread per Gaussian decides its proposal, finds or inserts the key and lowers the
//      slot's value to (proposal index + 1) with atomicMin: value 0 (an existing anchor)
//      always wins, otherwise the smallest proposal index does;
//   4. a proposal wins iff its slot's value is its own index + 1; the winners are listed in
//      index order by the order-preserving compaction of ogs_prune_anchors and written as
//      new anchor rows (voxel centre, level, voxel size, parent).
// Every float operation that decides a key or a threshold test is an explicit
// round-to-nearest step (product, sum, quotient), so the decisions are reproducible.
#include "internal.cuh"

namespace ogs {
namespace {

constexpr uint64_t kEmptyKey = ~0ull;
constexpr int kVoxBits = 20;
constexpr int kVoxLim = 1 << (kVoxBits - 1);
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;
constexpr int kMaxLevels = 15;           // levels 0..14: a key never equals kEmptyKey

struct GrowParams {
    float tau[16];        // growing threshold per level
    float voxel[16];      // voxel size per level
    int NL;
    int k;
    int next_level;       // 0: proposals stay at the Gaussian's own level
};

// Voxel key of point (x, y, z) on the grid of level L with spacing vs: the nearest grid point
// rint(p / vs) per axis (voxels centred on grid points, ties to even).  False if a coordinate
// leaves [-kVoxLim, kVoxLim) (or is not finite).
__device__ __forceinline__ bool voxel_key(float x, float y, float z, int L, float vs,
                                          uint64_t& key) {
    const float q[3] = {rintf(__fdiv_rn(x, vs)), rintf(__fdiv_rn(y, vs)), rintf(__fdiv_rn(z, vs))};
    uint64_t out = (uint64_t)L << 60;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!(q[a] >= -(float)kVoxLim && q[a] < (float)kVoxLim)) return false;
        out |= (uint64_t)((int)q[a] + kVoxLim) << (40 - 20 * a);
    }
    key = out;
    return true;
}

__device__ __forceinline__ int key_coord(uint64_t key, int a) {
    return (int)((key >> (40 - 20 * a)) & ((1u << kVoxBits) - 1)) - kVoxLim;
}

// 64-bit finaliser of MurmurHash3 (a published bit mixer): spreads nearby voxel keys.
__device__ __forceinline__ uint64_t mix64(uint64_t h) {
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    return h;
}

// Slot of `key`, inserted if absent.  The table has mask + 1 slots and is at most half full,
// so the probe ends long before its bound; returns kNoSlot only if every slot was visited.
__device__ __forceinline__ uint32_t find_or_insert(unsigned long long* keys, uint64_t mask,
                                                   uint64_t key) {
    uint64_t s = mix64(key) & mask;
    for (uint64_t p = 0; p <= mask; ++p) {
        const unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(keys + s);
        if (cur == key) return (uint32_t)s;
        if (cur == kEmptyKey) {
            const unsigned long long prev = atomicCAS(keys + s, kEmptyKey, key);
            if (prev == kEmptyKey || prev == key) return (uint32_t)s;
        }
        s = (s + 1) & mask;
    }
    return kNoSlot;
}

__global__ void grow_accumulate_kernel(const float* __restrict__ drec,
                                       const uint32_t* __restrict__ tiles,
                                       const uint32_t* __restrict__ sel_idx,
                                       const ogs_counts* counts, int k, float half_w,
                                       float half_h, float* __restrict__ acc,
                                       uint32_t* __restrict__ cnt) {
    const uint32_t G = counts->n_gaussians;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        if (tiles[g] == 0) continue;
        const uint32_t r = g / (uint32_t)k, i = g - r * (uint32_t)k;
        const size_t c = (size_t)sel_idx[r] * k + i;
        const float gx = __fmul_rn(drec[9 * (size_t)g], half_w);
        const float gy = __fmul_rn(drec[9 * (size_t)g + 1], half_h);
        acc[c] += __fsqrt_rn(__fmaf_rn(gy, gy, __fmul_rn(gx, gx)));
        cnt[c] += 1u;                 // an anchor appears once per view: no atomics
    }
}

__global__ void lod_bias_kernel(const uint8_t* __restrict__ level, const float* __restrict__ acc,
                                const uint32_t* __restrict__ cnt, int64_t N, GrowParams p,
                                float eps, float* __restrict__ dL) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        uint32_t c = 0;
        for (int i = 0; i < p.k; ++i) {
            s = __fadd_rn(s, acc[j * p.k + i]);
            c += cnt[j * p.k + i];
        }
        const int L = level[j];
        // p.tau holds the LOD-bias thresholds here
        if (c > 0 && L < p.NL && __fdiv_rn(s, (float)c) > p.tau[L]) dL[j] = __fadd_rn(dL[j], eps);
    }
}

__global__ void grow_clear(unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals,
                           uint64_t n) {
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (uint64_t)gridDim.x * blockDim.x) {
        keys[s] = kEmptyKey;
        vals[s] = 0xFFFFFFFFu;
    }
}

__global__ void grow_insert_anchors(const float* __restrict__ pos, const uint8_t* __restrict__ level,
                                    int64_t N, GrowParams p, unsigned long long* keys,
                                    uint32_t* vals, uint64_t mask, uint32_t* failed) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int L = level[j];
        uint64_t key;
        if (L >= p.NL ||
            !voxel_key(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], L, p.voxel[L], key))
            continue;
        const uint32_t s = find_or_insert(keys, mask, key);
        if (s == kNoSlot) { atomicExch(failed, 1u); continue; }
        vals[s] = 0u;                 // occupied by an anchor of this level
    }
}

__global__ void grow_propose(const float* __restrict__ pos, const uint8_t* __restrict__ level,
                             const float* __restrict__ offs, const float* __restrict__ lv,
                             const float* __restrict__ acc, const uint32_t* __restrict__ cnt,
                             int64_t NK, GrowParams p, unsigned long long* keys, uint32_t* vals,
                             uint64_t mask, uint32_t* __restrict__ slot_of, uint32_t* failed) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < NK;
         c += (int64_t)gridDim.x * blockDim.x) {
        slot_of[c] = kNoSlot;
        const uint32_t n = cnt[c];
        if (n == 0) continue;
        const int64_t j = c / p.k;
        const int L = level[j];
        if (L >= p.NL) continue;
        const float g = __fdiv_rn(acc[c], (float)n);
        int T;
        if (p.next_level && L + 1 < p.NL && g > p.tau[L + 1]) T = L + 1;
        else if (g > p.tau[L]) T = L;
        else continue;
        float mu[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            mu[a] = __fadd_rn(pos[3 * j + a], __fmul_rn(offs[3 * c + a], lv[3 * j + a]));
        uint64_t key;
        if (!voxel_key(mu[0], mu[1], mu[2], T, p.voxel[T], key)) continue;
        const uint32_t s = find_or_insert(keys, mask, key);
        if (s == kNoSlot) { atomicExch(failed, 1u); continue; }
        atomicMin(vals + s, (uint32_t)c + 1u);
        slot_of[c] = s;
    }
}

__global__ void grow_flags(const uint32_t* __restrict__ slot_of, const uint32_t* __restrict__ vals,
                           int64_t NK, uint32_t* __restrict__ win) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < NK;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = slot_of[c];
        win[c] = (s != kNoSlot && vals[s] == (uint32_t)c + 1u) ? 1u : 0u;
    }
}

__global__ void grow_emit(const uint32_t* __restrict__ list, const uint32_t* __restrict__ n_list,
                          const uint32_t* __restrict__ slot_of,
                          const unsigned long long* __restrict__ keys, GrowParams p,
                          int64_t max_new, const uint32_t* failed, float* __restrict__ new_pos,
                          uint8_t* __restrict__ new_level, float* __restrict__ new_lv,
                          uint32_t* __restrict__ parent, uint32_t* __restrict__ n_new) {
    // a table that ran full (impossible at half load) reports no growth rather than a
    // partial one
    const uint32_t need = *failed ? 0u : *n_list;
    const int64_t n = min((int64_t)need, max_new);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        n_new[0] = (uint32_t)n;
        n_new[1] = need;
    }
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = list[r];
        const uint64_t key = keys[slot_of[c]];
        const int T = (int)(key >> 60);
        const float vs = p.voxel[T];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            new_pos[3 * r + a] = __fmul_rn((float)key_coord(key, a), vs);
            new_lv[3 * r + a] = vs;
        }
        new_level[r] = (uint8_t)T;
        parent[r] = c / (uint32_t)p.k;
    }
}

struct GrowLayout {
    unsigned long long* keys;
    uint32_t* vals;
    uint32_t* slot_of;
    uint32_t* win;
    uint32_t* list;
    uint32_t* n_list;    // [0] winners, [1] table-full flag
    void* prune_scratch;
    size_t prune_bytes;
    uint64_t slots;
};

inline uint64_t table_slots(int64_t N, int32_t k) {
    const uint64_t need = 2ull * (uint64_t)(N > 0 ? N : 1) * (uint64_t)(k + 1);
    uint64_t s = 1024;
    while (s < need) s <<= 1;
    return s;
}

inline size_t grow_layout(int64_t N, int32_t k, void* base, GrowLayout* out) {
    Carver cv(base);
    GrowLayout g;
    const int64_t NK = (N > 0 ? N : 1) * (int64_t)k;
    g.slots = table_slots(N, k);
    g.keys = cv.take<unsigned long long>(g.slots);
    g.vals = cv.take<uint32_t>(g.slots);
    g.slot_of = cv.take<uint32_t>((size_t)NK);
    g.win = cv.take<uint32_t>((size_t)NK);
    g.list = cv.take<uint32_t>((size_t)NK);
    g.n_list = cv.take<uint32_t>(4);
    g.prune_bytes = ogs_prune_scratch_bytes(NK);
    g.prune_scratch = cv.take<unsigned char>(g.prune_bytes);
    if (out) *out = g;
    return cv.off + 256;
}

bool fill_params(GrowParams& p, const float* tau, const float* voxel, int32_t NL, int32_t k) {
    if (NL < 1 || NL > kMaxLevels || k < 1 || k > 16) return false;
    p.NL = NL;
    p.k = k;
    p.next_level = 1;
    for (int L = 0; L < 16; ++L) {
        p.tau[L] = L < NL && tau ? tau[L] : 0.f;
        p.voxel[L] = L < NL && voxel ? voxel[L] : 1.f;
        if (L < NL && voxel && !(voxel[L] > 0.f && voxel[L] < 3.0e38f)) return false;
    }
    return true;
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" ogs_status ogs_grow_accumulate(const float* drec, const uint32_t* tiles,
                                          const uint32_t* sel_idx, const ogs_counts* counts,
                                          int32_t k, int32_t width, int32_t height,
                                          float* grad_acc, uint32_t* grad_cnt, void* stream) {
    if (!drec || !tiles || !sel_idx || !counts || !grad_acc || !grad_cnt || k < 1 || k > 16 ||
        width <= 0 || height <= 0)
        return OGS_ERR_ARG;
    grow_accumulate_kernel<<<4 * kSmCount, 256, 0, (cudaStream_t)stream>>>(
        drec, tiles, sel_idx, counts, k, 0.5f * (float)width, 0.5f * (float)height, grad_acc,
        grad_cnt);
    return launch_status();
}

extern "C" ogs_status ogs_update_lod_bias(const uint8_t* level, const float* grad_acc,
                                          const uint32_t* grad_cnt, int64_t N, int32_t k,
                                          int32_t NL, const float* thr_bias, float eps, float* dL,
                                          void* stream) {
    if (!level || !grad_acc || !grad_cnt || !thr_bias || !dL || N < 0) return OGS_ERR_ARG;
    GrowParams p;
    if (!fill_params(p, thr_bias, nullptr, NL, k)) return OGS_ERR_ARG;
    if (N == 0) return OGS_OK;
    lod_bias_kernel<<<stride_grid(N, 256, 8), 256, 0, (cudaStream_t)stream>>>(level, grad_acc,
                                                                               grad_cnt, N, p,
                                                                               eps, dL);
    return launch_status();
}

extern "C" size_t ogs_grow_scratch_bytes(int64_t N, int32_t k) {
    if (N < 0 || k < 1) return 0;
    return grow_layout(N, k, nullptr, nullptr);
}

extern "C" ogs_status ogs_grow_anchors(const float* pos, const uint8_t* level, const float* offs,
                                       const float* lv, const float* grad_acc,
                                       const uint32_t* grad_cnt, int64_t N, int32_t k, int32_t NL,
                                       const float* tau, const float* voxel, int32_t next_level,
                                       float* new_pos, uint8_t* new_level, float* new_lv,
                                       uint32_t* parent, int64_t max_new, uint32_t* n_new,
                                       void* scratch, size_t scratch_bytes, void* stream) {
    if (!tau || !voxel || !n_new || !scratch || N < 0 || max_new < 0) return OGS_ERR_ARG;
    if (N > 0 && (!pos || !level || !offs || !lv || !grad_acc || !grad_cnt)) return OGS_ERR_ARG;
    if (max_new > 0 && (!new_pos || !new_level || !new_lv || !parent)) return OGS_ERR_ARG;
    GrowParams p;
    if (!fill_params(p, tau, voxel, NL, k)) return OGS_ERR_ARG;
    p.next_level = next_level != 0;
    if ((uint64_t)N * (uint64_t)k >= 0xFFFFFFFFull || table_slots(N, k) > (1ull << 31))
        return OGS_ERR_ARG;
    if (scratch_bytes < ogs_grow_scratch_bytes(N, k) || !aligned(scratch, 16)) return OGS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    GrowLayout g;
    grow_layout(N, k, scratch, &g);
    const int64_t NK = N * (int64_t)k;
    const uint64_t mask = g.slots - 1;
    if (cudaMemsetAsync(g.n_list, 0, 4 * sizeof(uint32_t), st) != cudaSuccess) return OGS_ERR_CUDA;
    uint32_t* failed = g.n_list + 1;
    grow_clear<<<stride_grid((int64_t)g.slots, 256, 8), 256, 0, st>>>(g.keys, g.vals, g.slots);
    if (N > 0) {
        grow_insert_anchors<<<stride_grid(N, 256, 8), 256, 0, st>>>(pos, level, N, p, g.keys,
                                                                    g.vals, mask, failed);
        grow_propose<<<stride_grid(NK, 256, 8), 256, 0, st>>>(pos, level, offs, lv, grad_acc,
                                                              grad_cnt, NK, p, g.keys, g.vals,
                                                              mask, g.slot_of, failed);
        grow_flags<<<stride_grid(NK, 256, 8), 256, 0, st>>>(g.slot_of, g.vals, NK, g.win);
        const ogs_status s = ogs_prune_anchors(g.win, NK, 1u, g.list, g.n_list, g.prune_scratch,
                                               g.prune_bytes, st);
        if (s != OGS_OK) return s;
    }
    grow_emit<<<stride_grid(max_new > 0 ? max_new : 1, 256, 8), 256, 0, st>>>(
        g.list, g.n_list, g.slot_of, g.keys, p, max_new, failed, new_pos, new_level, new_lv,
        parent, n_new);
    return launch_status();
}
