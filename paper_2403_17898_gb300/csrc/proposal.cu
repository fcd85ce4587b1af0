// Learned anchor-visibility proposal: a 3-layer MLP (37 -> 64 -> 64 -> 1, ReLU, ReLU,
// sigmoid) scores every anchor kept by the LOD rule from [f_v, L/(NL-1), unit viewing
// direction in the camera frame, ln(d/d_max)] and drops those whose keep probability is below
// p*, before any Gaussian is decoded.  Training labels are the renderer's own per-anchor maximum
// contribution (T * alpha) from ogs_blend_fwd.
//
// gate:  score pass (FP32: thread per selected anchor, weights in shared memory, outer-product
//        form so only the 40-wide input and 64 second-layer accumulators live in registers;
//        BF16: both hidden layers as tcgen05 MMAs over 128-anchor tiles; per-tile keep
//        counts) -> scan -> order-preserving scatter of the kept entries.
// train: thread per selected anchor: forward, BCE gradient dL/dz = (p - y)/M, backward;
//        weight gradients as per-block sums of outer products staged in shared memory,
//        written as partials and summed in a fixed order.
#include <cstring>

#include "gate_common.cuh"

namespace ogs {
namespace {

using namespace gate;

constexpr int kGateThreads = 128;
constexpr int kNetFloats = kPH * kPInPad + kPH + kPH * kPH + kPH + kPH + 4;   // smem image

struct PropArgs {
    const float* pos;
    const uint8_t* level;
    const float* feat;
    int NL;
    Cam cam;
    ogs_proposal net;
};

// Loads the network into shared memory: w1 [64][40] (zero padded), b1, w2t [64][64] (w2
// transposed: row o holds the weights that hidden-1 unit o feeds), b2, w3, b3.
__device__ void load_net(const ogs_proposal& n, float* s) {
    float* w1 = s;
    float* b1 = w1 + kPH * kPInPad;
    float* w2t = b1 + kPH;
    float* b2 = w2t + kPH * kPH;
    float* w3 = b2 + kPH;
    float* b3 = w3 + kPH;
    for (int e = threadIdx.x; e < kPH * kPInPad; e += blockDim.x) {
        const int o = e / kPInPad, i = e % kPInPad;
        w1[e] = i < kPIn ? n.w1[o * kPIn + i] : 0.f;
    }
    for (int e = threadIdx.x; e < kPH * kPH; e += blockDim.x) {
        const int o = e / kPH, i = e % kPH;
        w2t[e] = n.w2[i * kPH + o];
    }
    for (int e = threadIdx.x; e < kPH; e += blockDim.x) {
        b1[e] = n.b1[e];
        b2[e] = n.b2[e];
        w3[e] = n.w3[e];
    }
    if (threadIdx.x == 0) b3[0] = n.b3[0];
}

__device__ __forceinline__ void prop_input(const PropArgs& a, uint32_t j, float (&x)[kPInPad]) {
    prop_input_vals(a.feat + (size_t)j * 32, a.pos[3 * (size_t)j], a.pos[3 * (size_t)j + 1],
                    a.pos[3 * (size_t)j + 2], a.level[j], a.NL, a.cam, x);
}

__device__ __forceinline__ float prop_logit(const float* s, const float (&x)[kPInPad]) {
    const float* w1 = s;
    const float* b1 = w1 + kPH * kPInPad;
    const float* w2t = b1 + kPH;
    const float* b2 = w2t + kPH * kPH;
    const float* w3 = b2 + kPH;
    const float* b3 = w3 + kPH;
    float h2[kPH];
#pragma unroll
    for (int i = 0; i < kPH; ++i) h2[i] = b2[i];
#pragma unroll 1
    for (int o = 0; o < kPH; ++o) {
        const float4* row = reinterpret_cast<const float4*>(w1 + o * kPInPad);
        float acc = b1[o];
#pragma unroll
        for (int i = 0; i < kPInPad / 4; ++i) {
            const float4 w = row[i];
            acc = fmaf(w.x, x[4 * i], acc);
            acc = fmaf(w.y, x[4 * i + 1], acc);
            acc = fmaf(w.z, x[4 * i + 2], acc);
            acc = fmaf(w.w, x[4 * i + 3], acc);
        }
        const float h1 = fmaxf(acc, 0.f);
        const float4* col = reinterpret_cast<const float4*>(w2t + o * kPH);
#pragma unroll
        for (int i = 0; i < kPH / 4; ++i) {
            const float4 w = col[i];
            h2[4 * i] = fmaf(w.x, h1, h2[4 * i]);
            h2[4 * i + 1] = fmaf(w.y, h1, h2[4 * i + 1]);
            h2[4 * i + 2] = fmaf(w.z, h1, h2[4 * i + 2]);
            h2[4 * i + 3] = fmaf(w.w, h1, h2[4 * i + 3]);
        }
    }
    float z = b3[0];
#pragma unroll
    for (int i = 0; i < kPH; ++i) z = fmaf(w3[i], fmaxf(h2[i], 0.f), z);
    return z;
}

// score pass: p per selected anchor (scratch), keep counts per block, old M saved
__global__ void __launch_bounds__(kGateThreads) gate_score(PropArgs a, const uint32_t* sel_idx,
                                                           const ogs_counts* counts, float p_star,
                                                           float* p_out, uint32_t* block_count,
                                                           uint32_t* m_saved) {
    extern __shared__ __align__(16) float s[];
    __shared__ uint32_t wc[kGateThreads / 32];
    const uint32_t M = counts->n_selected;
    if (blockIdx.x == 0 && threadIdx.x == 0) *m_saved = M;
    const uint32_t r = blockIdx.x * kGateThreads + threadIdx.x;
    bool keep = false;
    if ((uint32_t)blockIdx.x * kGateThreads < M) {
        load_net(a.net, s);
        __syncthreads();
        if (r < M) {
            float x[kPInPad];
            prop_input(a, sel_idx[r], x);
            const float p = 1.0f / (1.0f + __expf(-prop_logit(s, x)));
            p_out[r] = p;
            keep = p >= p_star;
        }
    }
    const unsigned b = __ballot_sync(0xffffffffu, keep);
    if (lane_id() == 0) wc[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kGateThreads / 32; ++i) t += wc[i];
        block_count[blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------------------
// BF16 tensor-core scoring (tcgen05): 128 selected anchors per tile,
//   layer 1: D[128 x 64] = X[128 x 48] . W1^T   (37 inputs padded to 48)
//   layer 2: D[128 x 64] = H1[128 x 64] . W2^T  (reuses layer 1's TMEM columns)
// operands in shared memory (no-swizzle K-major core matrices), FP32 accumulators in TMEM;
// bias/ReLU epilogues and the final 64-wide dot product + sigmoid in FP32, one anchor per
// thread.  Same outputs as gate_score: p per entry, keep count per 128-entry tile.
// ---------------------------------------------------------------------------------------

constexpr int kGOffA = kGImgBytes;                       // A operand after the image
constexpr int kGSmem = kGOffA + kGABytes;
static_assert(kGOffA % 16 == 0, "bulk copy granularity");
static_assert(kGateThreads == 128, "one TMEM lane (anchor) per thread");

// Per call: the first kGPackCtas CTAs write the network image (BF16 operand tiles of W1 (K
// padded to 48) and W2 in the no-swizzle K-major core-matrix layout, then b1, b2, w3, b3 in
// FP32) to global scratch, one 8-element group or vector entry per thread; the other CTAs zero
// the tile status words and the ticket/done counters.
constexpr int kGPackThreads = 256;
constexpr int kGGroups1 = kPH * (kGK1 / 8), kGGroups2 = kPH * (kPH / 8);
constexpr int kGPackItems = kGGroups1 + kGGroups2 + 3 * kPH + 4;
constexpr int kGPackCtas = (kGPackItems + kGPackThreads - 1) / kGPackThreads;

__global__ void __launch_bounds__(kGPackThreads) gate_pack(ogs_proposal net, unsigned char* img,
                                                           unsigned long long* status,
                                                           int n_words) {
    pdl_wait();
    pdl_trigger();
    if (blockIdx.x < kGPackCtas) {
        const int e = blockIdx.x * kGPackThreads + threadIdx.x;
        float v[8];
        if (e < kGGroups1) {
            const int n = e / (kGK1 / 8), kc = e % (kGK1 / 8);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int kk = 8 * kc + i;
                v[i] = kk < kPIn ? net.w1[n * kPIn + kk] : 0.f;
            }
            gput8(img + kGOffB1, n, kc, kGK1, v);
        } else if (e < kGGroups1 + kGGroups2) {
            const int f = e - kGGroups1;
            const int n = f / (kPH / 8), kc = f % (kPH / 8);
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = net.w2[n * kPH + 8 * kc + i];
            gput8(img + kGOffB2, n, kc, kPH, v);
        } else if (e < kGPackItems) {
            const int f = e - kGGroups1 - kGGroups2;
            reinterpret_cast<float*>(img + kGOffVec)[f] =
                f < kPH ? net.b1[f] : f < 2 * kPH ? net.b2[f - kPH]
                : f < 3 * kPH ? net.w3[f - 2 * kPH] : f == 3 * kPH ? net.b3[0] : 0.f;
        }
        return;
    }
    const int nz = gridDim.x - kGPackCtas;
    for (int e = (blockIdx.x - kGPackCtas) * kGPackThreads + threadIdx.x; e < n_words;
         e += nz * kGPackThreads)
        status[e] = 0ull;
}

// Single pass: CTAs take 128-entry tiles by ticket, score them on the tensor cores, publish
// the tile's keep count, find its output offset by look-back and write the kept entries in
// order.  The last CTA to finish (when every CTA has read the input count) publishes the new
// counts.
__global__ void __launch_bounds__(kGateThreads, 5) gate_tc(PropArgs a, const uint32_t* sel_in,
                                                           const float* w_in, int k,
                                                           ogs_counts* counts, float p_star,
                                                           float* p_out, uint32_t* sel_out,
                                                           float* w_out,
                                                           const unsigned char* img,
                                                           unsigned long long* status,
                                                           uint32_t* sync_words) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t wbar;
    __shared__ uint32_t tmem_base;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t wc[kGateThreads / 32];
    unsigned char* sA1 = sm + kGOffA;
    const int t = threadIdx.x, w = t >> 5;
    const uint32_t M = counts->n_selected;
    const uint32_t ntiles = (M + 127) / 128;
    uint32_t* ticket = sync_words;
    uint32_t* done = sync_words + 1;

    if (blockIdx.x < ntiles) {                   // uniform: CTAs with work own TMEM
        if (t == 0) {
            tc::mbar_init(&mbar, 1);
            tc::mbar_init(&wbar, 1);
            tc::mbar_expect_tx(&wbar, kGImgBytes);
            tc::bulk_load(sm, img, kGImgBytes, &wbar);   // lands while the inputs are gathered
        }
        if (w == 0) {
            tc::tmem_alloc(&tmem_base, kGTmemCols);
            tc::tmem_relinquish();
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        const uint32_t tbase = tmem_base;
        uint32_t phase = 0;
        bool aborted = false;
        bool have_net = false;

        for (;;) {
            if (t == 0) s_tile = atomicAdd(ticket, 1u);
            __syncthreads();
            const uint32_t tile = s_tile;
            if (tile >= ntiles) break;
            const uint32_t r = tile * 128 + t;
            const bool valid = r < M;
            {
                float x[kPInPad];
                if (valid) {
                    prop_input(a, sel_in[r], x);
                } else {
#pragma unroll
                    for (int i = 0; i < kPInPad; ++i) x[i] = 0.f;
                }
                put_input_row(sA1, t, x);
            }
            if (!have_net) {                          // the network image, once per CTA
                have_net = true;
                if (!tc::mbar_wait(&wbar, 0, kGWaitLimit)) {
                    // copy still in flight: wait once more (bounded) before anyone leaves
                    if (t == 0) atomicExch(&counts->timeout, 1u);
                    tc::mbar_wait(&wbar, 0, kGWaitLimit);
                }
            }
            float z;
            if (!gate_hidden(sA1, sm, tbase, &mbar, phase, z)) {
                aborted = true;
                if (t == 0) store_status(status + tile, kFlagPrefix);   // let successors finish
                break;
            }
            bool keep = false;
            if (valid) {
                const float p = keep_prob(z);
                if (p_out) p_out[r] = p;
                keep = p >= p_star;
            }
            const unsigned b = __ballot_sync(0xffffffffu, keep);
            if (lane_id() == 0) wc[w] = __popc(b);
            // also orders this tile's TMEM reads before the next tile's MMAs
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            const unsigned long long agg = wc[0] + wc[1] + wc[2] + wc[3];
            const unsigned long long excl =
                block_tile_offset<kGateThreads>(status, tile, agg, &counts->timeout);
            if (keep) {
                uint32_t wpre = 0;
                for (int i = 0; i < w; ++i) wpre += wc[i];
                const unsigned long long o = excl + wpre + __popc(b & lanemask_lt());
                sel_out[o] = sel_in[r];
                w_out[o] = w_in[r];
            }
        }
        if (aborted) {
            if (t == 0) atomicExch(&counts->timeout, 1u);
            tc::mbar_wait(&mbar, phase, kGWaitLimit);
        }
        if (!have_net) tc::mbar_wait(&wbar, 0, kGWaitLimit);   // no tile taken: let the copy land
        tc::fence_before_sync();
        __syncthreads();
        if (w == 0) tc::tmem_dealloc(tbase, kGTmemCols);
    }
    // the last CTA to finish publishes the kept count (every CTA has read M by then)
    if (t == 0) {
        __threadfence();
        if (atomicAdd(done, 1u) == gridDim.x - 1) {
            __threadfence();
            const uint32_t kept =
                ntiles ? (uint32_t)(load_status(status + ntiles - 1) & kValMask) : 0u;
            counts->n_selected = kept;
            counts->n_gaussians = kept * (uint32_t)k;
        }
    }
}

__global__ void __launch_bounds__(1024) gate_scan(uint32_t* block_count, int nb_cap, int k,
                                                  const uint32_t* m_saved, ogs_counts* counts) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    // only the tiles that hold entries were scored
    const int nb = min(nb_cap, (int)((*m_saved + kGateThreads - 1) / kGateThreads));
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const uint32_t v = b < nb ? block_count[b] : 0;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (unsigned)o) x += y;
        }
        if (lane_id() == 31) ws[threadIdx.x >> 5] = x;
        __syncthreads();
        uint32_t wpre = 0, tot = 0;
        for (int q = 0; q < 32; ++q) {
            wpre += (q < (int)(threadIdx.x >> 5)) ? ws[q] : 0;
            tot += ws[q];
        }
        const uint32_t excl = carry + wpre + x - v;
        if (b < nb) block_count[b] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        counts->n_selected = carry;
        counts->n_gaussians = carry * (uint32_t)k;
    }
}

__global__ void __launch_bounds__(kGateThreads) gate_scatter(
    const uint32_t* sel_in, const float* w_in, const float* p, float p_star,
    const uint32_t* m_saved, const uint32_t* block_off, uint32_t* sel_out, float* w_out) {
    __shared__ uint32_t wc[kGateThreads / 32];
    const uint32_t M = *m_saved;
    const uint32_t r = blockIdx.x * kGateThreads + threadIdx.x;
    const bool keep = r < M && p[r] >= p_star;
    const unsigned b = __ballot_sync(0xffffffffu, keep);
    if (lane_id() == 0) wc[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    uint32_t wpre = 0;
    for (int i = 0; i < (int)(threadIdx.x >> 5); ++i) wpre += wc[i];
    if (keep) {
        const uint32_t o = block_off[blockIdx.x] + wpre + __popc(b & lanemask_lt());
        sel_out[o] = sel_in[r];
        w_out[o] = w_in[r];
    }
}

// ---------------------------------------------------------------------------------------
// training
// ---------------------------------------------------------------------------------------

constexpr int kTrThreads = 64;
// gradient layout (flat): dw1 [64][37] | db1 [64] | dw2 [64][64] | db2 [64] | dw3 [64] | db3
constexpr int kGW1 = 0;
constexpr int kGB1 = kGW1 + kPH * kPIn;
constexpr int kGW2 = kGB1 + kPH;
constexpr int kGB2 = kGW2 + kPH * kPH;
constexpr int kGW3 = kGB2 + kPH;
constexpr int kGB3 = kGW3 + kPH;
constexpr int kGrads = kGB3 + 1;
constexpr int kTrBlocks = 2 * kSmCount;

struct TrainArgs {
    PropArgs pa;
    const uint32_t* sel_idx;
    const ogs_counts* counts;
    const uint32_t* maxc;
    uint32_t tau_bits;
    float pos_weight;
    float* partial;
    float* loss;
};

__global__ void __launch_bounds__(kTrThreads) prop_train_kernel(TrainArgs a) {
    extern __shared__ __align__(16) float s[];
    float* net = s;                                  // kNetFloats
    float* acc = net + kNetFloats;                   // kGrads
    float* sX = acc + ((kGrads + 3) / 4) * 4;        // [T][40]
    float* sH1 = sX + kTrThreads * kPInPad;          // [T][64]
    float* sH2 = sH1 + kTrThreads * kPH;             // [T][64]  relu(a2)
    float* sD1 = sH2 + kTrThreads * kPH;             // [T][64]  dL/da1
    float* sD2 = sD1 + kTrThreads * kPH;             // [T][64]  dL/da2
    float* sDZ = sD2 + kTrThreads * kPH;             // [T]
    load_net(a.pa.net, net);
    for (int e = threadIdx.x; e < kGrads; e += blockDim.x) acc[e] = 0.f;
    __syncthreads();
    const float* w1 = net;
    const float* b1 = w1 + kPH * kPInPad;
    const float* w2t = b1 + kPH;
    const float* b2 = w2t + kPH * kPH;
    const float* w3 = b2 + kPH;
    const float* b3 = w3 + kPH;
    const uint32_t M = a.counts->n_selected;
    const float invM = M ? 1.0f / (float)M : 0.f;
    const int t = threadIdx.x;
    float lsum = 0.f;
    for (uint32_t base = blockIdx.x * kTrThreads; base < M; base += gridDim.x * kTrThreads) {
        const uint32_t r = base + t;
        const bool valid = r < M;
        float x[kPInPad];
        uint32_t j = 0;
        if (valid) {
            j = a.sel_idx[r];
            prop_input(a.pa, j, x);
        } else {
#pragma unroll
            for (int i = 0; i < kPInPad; ++i) x[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < kPInPad; ++i) sX[t * kPInPad + i] = x[i];
        // forward, keeping a1 sign in sD1 temporarily and h1 in sH1
        float a2[kPH];
#pragma unroll
        for (int i = 0; i < kPH; ++i) a2[i] = b2[i];
        for (int o = 0; o < kPH; ++o) {
            float acc1 = b1[o];
#pragma unroll
            for (int i = 0; i < kPInPad; ++i) acc1 = fmaf(w1[o * kPInPad + i], x[i], acc1);
            const float h1 = fmaxf(acc1, 0.f);
            sH1[t * kPH + o] = h1;
            sD1[t * kPH + o] = acc1 > 0.f ? 1.f : 0.f;
#pragma unroll
            for (int i = 0; i < kPH; ++i) a2[i] = fmaf(w2t[o * kPH + i], h1, a2[i]);
        }
        float z = b3[0];
#pragma unroll
        for (int i = 0; i < kPH; ++i) {
            const float h2 = fmaxf(a2[i], 0.f);
            sH2[t * kPH + i] = h2;
            z = fmaf(w3[i], h2, z);
        }
        const float p = 1.0f / (1.0f + __expf(-z));
        float dz = 0.f;
        if (valid) {
            const float y = a.maxc[j] >= a.tau_bits ? 1.f : 0.f;
            const float wy = y > 0.f ? a.pos_weight : 1.f;
            dz = wy * (p - y) * invM;
            // BCE with the log-sigmoid written stably: -y z + log(1 + e^z)
            const float sp = z > 0.f ? z + log1pf(__expf(-z)) : log1pf(__expf(z));
            lsum += wy * (sp - y * z) * invM;
        }
        sDZ[t] = dz;
#pragma unroll
        for (int i = 0; i < kPH; ++i) sD2[t * kPH + i] = a2[i] > 0.f ? dz * w3[i] : 0.f;
        // dL/da1 = (W2^T dL/da2) * relu'(a1)
        for (int o = 0; o < kPH; ++o) {
            float g = 0.f;
#pragma unroll
            for (int i = 0; i < kPH; ++i) g = fmaf(w2t[o * kPH + i], sD2[t * kPH + i], g);
            sD1[t * kPH + o] *= g;
        }
        __syncthreads();
        const int nv = (int)min((uint32_t)kTrThreads, M - base);
        for (int e = t; e < kPH * kPIn; e += kTrThreads) {
            const int o = e / kPIn, i = e % kPIn;
            float sum = 0.f;
            for (int q = 0; q < nv; ++q) sum = fmaf(sD1[q * kPH + o], sX[q * kPInPad + i], sum);
            acc[kGW1 + e] += sum;
        }
        for (int e = t; e < kPH * kPH; e += kTrThreads) {
            const int o = e / kPH, i = e % kPH;
            float sum = 0.f;
            for (int q = 0; q < nv; ++q) sum = fmaf(sD2[q * kPH + o], sH1[q * kPH + i], sum);
            acc[kGW2 + e] += sum;
        }
        for (int e = t; e < kPH; e += kTrThreads) {
            float s1 = 0.f, s2 = 0.f, s3 = 0.f;
            for (int q = 0; q < nv; ++q) {
                s1 += sD1[q * kPH + e];
                s2 += sD2[q * kPH + e];
                s3 = fmaf(sDZ[q], sH2[q * kPH + e], s3);
            }
            acc[kGB1 + e] += s1;
            acc[kGB2 + e] += s2;
            acc[kGW3 + e] += s3;
        }
        if (t == 0) {
            float s0 = 0.f;
            for (int q = 0; q < nv; ++q) s0 += sDZ[q];
            acc[kGB3] += s0;
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane_id() == 0 && a.loss) atomicAdd(a.loss, lsum);
    float* out = a.partial + (size_t)blockIdx.x * kGrads;
    for (int e = t; e < kGrads; e += kTrThreads) out[e] = acc[e];
}

// dloss (device, may be null = 1): gradient of the caller's objective with respect to the BCE
// loss, the chain-rule factor of every weight gradient
__global__ void prop_reduce(const float* __restrict__ partial, int nblocks, ogs_proposal g,
                            const float* __restrict__ dloss) {
    const float scale = dloss ? *dloss : 1.0f;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kGrads; e += gridDim.x * blockDim.x) {
        float sum = 0.f;
        for (int b = 0; b < nblocks; ++b) sum += partial[(size_t)b * kGrads + e];
        sum *= scale;
        float* dst;
        if (e < kGB1) dst = const_cast<float*>(g.w1) + (e - kGW1);
        else if (e < kGW2) dst = const_cast<float*>(g.b1) + (e - kGB1);
        else if (e < kGB2) dst = const_cast<float*>(g.w2) + (e - kGW2);
        else if (e < kGW3) dst = const_cast<float*>(g.b2) + (e - kGB2);
        else if (e < kGB3) dst = const_cast<float*>(g.w3) + (e - kGW3);
        else dst = const_cast<float*>(g.b3);
        *dst += sum;
    }
}

size_t train_smem() {
    return sizeof(float) * (kNetFloats + ((kGrads + 3) / 4) * 4 +
                            kTrThreads * (kPInPad + 4 * kPH + 1));
}

bool net_ok(const ogs_proposal* n) {
    return n && n->w1 && n->b1 && n->w2 && n->b2 && n->w3 && n->b3;
}

}  // namespace
}  // namespace ogs

using namespace ogs;

ogs_status ogs::gate::pack_image(const ogs_proposal& net, unsigned char* img,
                                 unsigned long long* status, int n_words, cudaStream_t st) {
    const int nz = n_words > 0 ? (n_words + 1023) / 1024 : 0;
    launch_pdl(gate_pack, dim3(kGPackCtas + nz), dim3(kGPackThreads), 0, st,
               net, img, status, n_words);
    return launch_status();
}

extern "C" size_t ogs_proposal_gate_scratch_bytes(int64_t sel_cap) {
    int64_t nb = (sel_cap + kGateThreads - 1) / kGateThreads;
    if (nb < 1) nb = 1;
    Carver cv(nullptr);
    cv.take<float>(sel_cap > 0 ? sel_cap : 1);
    cv.take<unsigned long long>(nb + 1);   // per-tile counts (FP32 form) or status words
    cv.take<uint32_t>(1);
    cv.take<unsigned char>(kGImgBytes);    // BF16 network image (tensor-core form)
    return cv.off + 256;
}

namespace {

ogs_status proposal_gate_impl(bool tensor_cores, const float* pos, const uint8_t* level,
                              const float* feat, int64_t N, int32_t NL, int32_t k,
                              const ogs_camera* cam, const ogs_proposal* net, float p_star,
                              const uint32_t* sel_in, const float* w_in, int64_t sel_cap,
                              ogs_counts* counts, uint32_t* sel_out, float* w_out, float* p_out,
                              void* scratch, size_t scratch_bytes, void* stream) {
    if (!pos || !level || !feat || !cam || !net_ok(net) || !sel_in || !w_in || !counts ||
        !sel_out || !w_out || !scratch)
        return OGS_ERR_ARG;
    if (N < 0 || NL < 1 || k < 1 || sel_cap < 0 || sel_in == sel_out) return OGS_ERR_ARG;
    if (scratch_bytes < ogs_proposal_gate_scratch_bytes(sel_cap) || !aligned(scratch, 16) ||
        !aligned(feat, 16))
        return OGS_ERR_ARG;
    if (sel_cap == 0) return OGS_OK;
    Carver cv(scratch);
    float* p = cv.take<float>(sel_cap);
    const int nb = (int)((sel_cap + kGateThreads - 1) / kGateThreads);
    uint32_t* block = reinterpret_cast<uint32_t*>(cv.take<unsigned long long>(nb + 1));
    uint32_t* m_saved = cv.take<uint32_t>(1);
    unsigned char* img = cv.take<unsigned char>(kGImgBytes);
    PropArgs a{pos, level, feat, NL, make_cam(*cam), *net};
    cudaStream_t st = (cudaStream_t)stream;
    if (tensor_cores) {
        // single pass: tile status words + ticket and done counters, zeroed by gate_pack
        // together with the network image
        unsigned long long* status = reinterpret_cast<unsigned long long*>(block);
        uint32_t* sync_words = reinterpret_cast<uint32_t*>(status + nb);
        if (gate::pack_image(*net, img, status, nb + 1, st) != OGS_OK) return OGS_ERR_CUDA;
        const int grid = nb < 5 * kSmCount ? nb : 5 * kSmCount;
        gate_tc<<<grid, kGateThreads, kGSmem, st>>>(a, sel_in, w_in, k, counts, p_star, p_out,
                                                    sel_out, w_out, img, status, sync_words);
        return launch_status();
    }
    const size_t smem = sizeof(float) * kNetFloats;
    gate_score<<<nb, kGateThreads, smem, st>>>(a, sel_in, counts, p_star, p, block, m_saved);
    gate_scan<<<1, 1024, 0, st>>>(block, nb, k, m_saved, counts);
    gate_scatter<<<nb, kGateThreads, 0, st>>>(sel_in, w_in, p, p_star, m_saved, block, sel_out, w_out);
    if (p_out)
        cudaMemcpyAsync(p_out, p, sizeof(float) * sel_cap, cudaMemcpyDeviceToDevice, st);
    return launch_status();
}

}  // namespace

extern "C" ogs_status ogs_proposal_gate(const float* pos, const uint8_t* level, const float* feat,
                                        int64_t N, int32_t NL, int32_t k, const ogs_camera* cam,
                                        const ogs_proposal* net, float p_star,
                                        const uint32_t* sel_in, const float* w_in, int64_t sel_cap,
                                        ogs_counts* counts, uint32_t* sel_out, float* w_out,
                                        float* p_out, void* scratch, size_t scratch_bytes,
                                        void* stream) {
    return proposal_gate_impl(false, pos, level, feat, N, NL, k, cam, net, p_star, sel_in, w_in,
                              sel_cap, counts, sel_out, w_out, p_out, scratch, scratch_bytes,
                              stream);
}

extern "C" ogs_status ogs_proposal_gate_bf16(const float* pos, const uint8_t* level,
                                             const float* feat, int64_t N, int32_t NL, int32_t k,
                                             const ogs_camera* cam, const ogs_proposal* net,
                                             float p_star, const uint32_t* sel_in,
                                             const float* w_in, int64_t sel_cap,
                                             ogs_counts* counts, uint32_t* sel_out, float* w_out,
                                             float* p_out, void* scratch, size_t scratch_bytes,
                                             void* stream) {
    return proposal_gate_impl(true, pos, level, feat, N, NL, k, cam, net, p_star, sel_in, w_in,
                              sel_cap, counts, sel_out, w_out, p_out, scratch, scratch_bytes,
                              stream);
}

extern "C" size_t ogs_proposal_train_scratch_bytes(void) {
    return sizeof(float) * (size_t)kTrBlocks * kGrads + 256;
}

extern "C" ogs_status ogs_proposal_train(const float* pos, const uint8_t* level, const float* feat,
                                         int64_t N, int32_t NL, const ogs_camera* cam,
                                         const ogs_proposal* net, const uint32_t* sel_idx,
                                         const ogs_counts* counts, const uint32_t* maxc,
                                         float tau, float pos_weight, const ogs_proposal* grads,
                                         float* loss, const float* dloss,
                                         void* scratch, size_t scratch_bytes, void* stream) {
    if (!pos || !level || !feat || !cam || !net_ok(net) || !sel_idx || !counts || !maxc ||
        !net_ok(grads) || !scratch)
        return OGS_ERR_ARG;
    if (N < 0 || NL < 1 || !(tau >= 0.f) || !(pos_weight > 0.f)) return OGS_ERR_ARG;
    if (scratch_bytes < ogs_proposal_train_scratch_bytes() || !aligned(scratch, 16) ||
        !aligned(feat, 16))
        return OGS_ERR_ARG;
    const size_t smem = train_smem();
    if (cudaFuncSetAttribute(prop_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return OGS_ERR_CUDA;
    uint32_t tau_bits;
    memcpy(&tau_bits, &tau, sizeof tau_bits);
    TrainArgs a{{pos, level, feat, NL, make_cam(*cam), *net}, sel_idx, counts, maxc, tau_bits,
                pos_weight, (float*)scratch, loss};
    cudaStream_t st = (cudaStream_t)stream;
    prop_train_kernel<<<kTrBlocks, kTrThreads, smem, st>>>(a);
    prop_reduce<<<(kGrads + 255) / 256, 256, 0, st>>>((const float*)scratch, kTrBlocks, *grads,
                                                       dloss);
    return launch_status();
}
