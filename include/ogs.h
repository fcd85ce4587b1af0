/*
 * ogs.h — C ABI of the GB300 (sm_103a) Octree-GS LOD renderer hot path.
 *
 * One view (or one training step) runs as a chain of stream-ordered calls:
 *
 *   ogs_lod_select   anchors -> selected anchor indices + opacity weights   (Sec. 4.1.3)
 *   ogs_decode       selected anchors -> k neural Gaussians each            (Sec. 3.2)
 *   ogs_project_bin  Gaussians -> 2D screen records, depth keys, tile rects (Sec. 3.1)
 *   ogs_sort         per-tile Gaussian lists in front-to-back order         (Sec. 3.1)
 *   ogs_blend_fwd    per-pixel front-to-back alpha blending                 (Sec. 3.1, Eq. 2)
 *   ogs_blend_bwd, ogs_project_bwd, ogs_decode_bwd   analytic backward (training)
 *   ogs_explicit_gaussians(_bwd)   explicit per-anchor Gaussians in place of decoding
 *   ogs_count_selected, ogs_prune_anchors, ogs_gather_rows   view-frequency pruning
 *   ogs_opacity_accumulate, ogs_prune_by_opacity   average-opacity pruning (Sec. 4.2.2)
 *   ogs_grow_accumulate, ogs_update_lod_bias, ogs_grow_anchors   anchor growing (Sec. 4.2.1)
 *
 * Conventions shared by every entry point
 *   - Every pointer argument is a DEVICE pointer unless its comment says "host".  All device
 *     memory is owned by the caller; the library never allocates or frees device memory and
 *     keeps no global state.  Scratch space is passed in by the caller; its size comes from
 *     the matching *_scratch_bytes() query.
 *   - `stream` is a cudaStream_t passed as void*.  Every call only enqueues work on it and
 *     returns without synchronising; outputs are valid once the stream reaches that point.
 *   - Counts produced on the device (selected anchors, Gaussians, pairs) stay on the device in
 *     an ogs_counts record that later calls read, so a frame needs no host round trip.  Buffer
 *     capacities are passed from the host; a count that exceeds its capacity sets a bit in
 *     ogs_counts.overflow, records the size that would have been needed, and the affected
 *     stage writes only what fits (the caller grows the buffer and reruns the frame).
 *   - Return value: OGS_OK, or OGS_ERR_ARG for a null pointer / bad size / misaligned pointer
 *     detected on the host before anything is enqueued, or OGS_ERR_CUDA when a launch fails.
 *     Errors found on the device (capacity, expired waits, non-finite values) stay in device
 *     words; ogs_counts_status turns a read-back copy into a status.  No call throws, traps
 *     or exits.
 *   - Arrays are C-contiguous; "f32[N][3]" means N rows of 3 floats.
 *
 * Camera model: world point p has camera coordinates R (p - campos) (x right, y down, z
 * forward); its pixel is (fx x/z + cx, fy y/z + cy) with pixel (i, j) centred on integer
 * coordinates.  Tiles are 16x16 pixels; the tile grid is ceil(W/16) x ceil(H/16).
 */
#ifndef OGS_H
#define OGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ogs_status {
    OGS_OK = 0,
    OGS_ERR_ARG = 1,       /* invalid argument, nothing enqueued */
    OGS_ERR_CAPACITY = 2,  /* a capacity was too small (host check, or ogs_counts.overflow) */
    OGS_ERR_TIMEOUT = 3,   /* a bounded device-side wait expired (see ogs_counts.timeout) */
    OGS_ERR_CUDA = 4,      /* a CUDA launch or API call failed */
    OGS_ERR_NONFINITE = 5  /* ogs_scan_nonfinite found a NaN or infinity */
} ogs_status;

/* Host-side camera, passed by pointer and copied at call time. */
typedef struct ogs_camera {
    float R[9];        /* world -> camera rotation, row-major */
    float campos[3];   /* camera centre, world */
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear;       /* near plane, camera z (0.2 by convention) */
    float d_max;       /* reference distance of the LOD rule */
    float s;           /* focal scale factor of the LOD rule */
    float pad;
} ogs_camera;

/* Device-resident counters of one frame.  The caller zeroes the record before
 * ogs_lod_select (cudaMemsetAsync); the kernels fill it in. */
typedef struct ogs_counts {
    uint32_t n_selected;       /* M, anchors kept by ogs_lod_select (<= its capacity) */
    uint32_t n_gaussians;      /* M * k */
    uint32_t n_pairs;          /* P, (tile, Gaussian) pairs (<= pair capacity) */
    uint32_t overflow;         /* bit 0: selection capacity, bit 1: pair capacity */
    uint32_t need_selected;    /* selection size that was needed */
    uint32_t need_pairs;       /* pair count that was needed */
    uint32_t timeout;          /* nonzero if a bounded wait expired */
    uint32_t reserved;         /* zero (pads the record to 32 bytes) */
} ogs_counts;

/* Decoder weights (device, f32), layout of the paper's three attribute MLPs (Sec. 3.2,
 * Eq. mlp): input z = [f_v (F), (x_v - campos)/|x_v - campos| (3), |x_v - campos| (1)],
 * Din = F + 4, hidden H = 32, ReLU.
 *   w1  f32[3][H][Din], b1 f32[3][H]   (0 = opacity, 1 = colour, 2 = covariance)
 *   w2_op  f32[k][H],   b2_op  f32[k]    opacity_i  = w * tanh(.)   (dropped if <= 0)
 *   w2_col f32[3k][H],  b2_col f32[3k]   colour_i   = sigmoid(rows 3i..3i+2)
 *   w2_cov f32[7k][H],  b2_cov f32[7k]   scale_i    = l_v * sigmoid(rows 7i..7i+2),
 *                                        quat_i (w,x,y,z) = normalise(rows 7i+3..7i+6)
 * Appearance codes (Sec. 4.4, optional, A = 0 disables them): anchor j carries a learnable
 * code a_j of A <= 8 values that only the colour decoder sees; its first layer adds
 * w1_app a_j to the hidden pre-activations (w1_app f32[H][A], app f32[N][A]; no alignment
 * requirement; A > 0 needs both).  When an ogs_mlp passes gradients (dmlp of ogs_decode_bwd),
 * w1_app and app are the gradient arrays of the same shapes (ACCUMULATED: +=). */
typedef struct ogs_mlp {
    const float* w1;
    const float* b1;
    const float* w2_op;
    const float* b2_op;
    const float* w2_col;
    const float* b2_col;
    const float* w2_cov;
    const float* b2_cov;
    int32_t F;          /* feature width (32) */
    int32_t H;          /* hidden width, must be 32 */
    int32_t k;          /* Gaussians per anchor (1..16) */
    int32_t A;          /* appearance code width (0..8); 0: no codes, w1_app/app unused */
    const float* w1_app;  /* f32[H][A] colour decoder's first-layer weights of the code */
    const float* app;     /* f32[N][A] per-anchor appearance codes */
} ogs_mlp;

/* Neural-Gaussian structure of arrays (device, f32); Gaussian g = r*k + i belongs to the r-th
 * selected anchor.  means are CAMERA-RELATIVE (mu - campos, world axes) when written by
 * ogs_decode: subtracting the camera centre before rounding keeps FP32 positions accurate at
 * city scale. */
typedef struct ogs_gaussians {
    float* means;    /* f32[G][3] */
    float* scales;   /* f32[G][3] */
    float* quats;    /* f32[G][4] unit quaternion (w, x, y, z) */
    float* opac;     /* f32[G]    opacity; <= 0 marks a dropped Gaussian */
    float* colors;   /* f32[G][3] */
} ogs_gaussians;

/* Screen-space record of one Gaussian (48 bytes, 16-byte aligned), written by
 * ogs_project_bin:  {u, v, conic_a, conic_b}, {conic_c, opacity, r, g},
 * {b, depth, radius, p_skip}.  The 2D falloff at pixel offset (dx, dy) = (u - px, v - py) is
 * G = exp(power), power = -0.5 (a dx^2 + c dy^2) - b dx dy; p_skip = -ln(255 opacity), so
 * alpha = opacity G < 1/255 exactly when power < p_skip (the blend tests the exponent before
 * evaluating exp; forward and backward use the same test). */
typedef struct ogs_rec2d {
    float u, v, ca, cb;
    float cc, o, cr, cg;
    float cbl, depth, radius, p_skip;
} ogs_rec2d;

/* ---------------------------------------------------------------------------------------
 * ogs_lod_select — Sec. 4.1.3, Eq. for L_hat and the inference-time opacity blending.
 * For each anchor j: d = |pos_j - campos|, L* = clamp(log2(d_max/(d s)) + dL_j, 0, NL-1),
 * L_hat = floor(L*).  The anchor is kept with weight 1 if level_j <= L_hat; with infer != 0
 * it is also kept with weight L* - L_hat if level_j == L_hat + 1 and that weight is > 0.
 * Only anchors whose centre is in front of the near plane and within 1.3x the half field of
 * view are considered.  Output is order-preserving: sel_idx ascending.
 *   pos f32[N][3], level u8[N], dL f32[N]      anchor SoA (inputs)
 *   sel_idx u32[sel_cap], sel_w f32[sel_cap]   outputs; counts->n_selected = M,
 *                                              counts->n_gaussians = M * k
 *   scratch: ogs_lod_select_scratch_bytes(N) bytes, 16-byte aligned.
 * ------------------------------------------------------------------------------------- */
size_t ogs_lod_select_scratch_bytes(int64_t N);
ogs_status ogs_lod_select(const float* pos, const uint8_t* level, const float* dL, int64_t N,
                          int32_t NL, int32_t k, const ogs_camera* cam /* host */,
                          int32_t infer, uint32_t* sel_idx, float* sel_w, int64_t sel_cap,
                          ogs_counts* counts, void* scratch, size_t scratch_bytes,
                          void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_decode — Sec. 3.2, Eq. offsets (mu_i = x_v + O_i * l_v, elementwise) and Eq. mlp.
 * FP32 arithmetic.  Reads M from counts->n_selected; writes Gaussians 0 .. M*k-1.
 *   pos f32[N][3], feat f32[N][F], offs f32[N][k][3], lv f32[N][3]   anchor SoA
 *   sel_idx/sel_w from ogs_lod_select; sel_cap = their capacity
 *   out: Gaussian SoA with room for sel_cap * k Gaussians (means camera-relative)
 *   mlp->A > 0: the colour decoder also sees the anchor's appearance code (Sec. 4.4)
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_decode(const float* pos, const float* feat, const float* offs, const float* lv,
                      int64_t N, const ogs_mlp* mlp /* host struct of device ptrs */,
                      const ogs_camera* cam /* host */, const uint32_t* sel_idx,
                      const float* sel_w, int64_t sel_cap, const ogs_counts* counts,
                      const ogs_gaussians* out /* host struct of device ptrs */, void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_decode_bf16 — ogs_decode on the tensor cores: both decoder layers as BF16 x BF16 MMAs
 * with FP32 accumulation (tcgen05, accumulators in tensor memory); inputs and hidden
 * activations are rounded to BF16, everything after the GEMMs (biases, activations,
 * normalisation, positions) is FP32.  Same arguments, layout and outputs as ogs_decode;
 * an appearance code enters layer 1 as BF16 K columns 40..47 (the input's zero padding).
 * counts is written only if a bounded internal wait expires (counts->timeout = 1, outputs
 * of the remaining anchors not written).
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_decode_bf16(const float* pos, const float* feat, const float* offs,
                           const float* lv, int64_t N, const ogs_mlp* mlp /* host struct */,
                           const ogs_camera* cam /* host */, const uint32_t* sel_idx,
                           const float* sel_w, int64_t sel_cap, ogs_counts* counts,
                           const ogs_gaussians* out /* host struct */, void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_project_bin — Sec. 3.1: Sigma = R(q) S S^T R(q)^T (Eq. 1), EWA projection
 * Sigma' = J W Sigma W^T J^T + 0.3 I (J with x/z, y/z clamped to 1.3x the half-fov),
 * conic = Sigma'^-1, radius r = 3 sqrt(lambda_max), lambda_max = mid + sqrt(max(0.1,
 * mid^2 - det)), tile rectangle of the tiles holding a pixel centre inside [u-r, u+r] x
 * [v-r, v+r].  A Gaussian is culled (rect empty, tiles 0, depth key 0xFFFFFFFF) when its
 * opacity is <= 0, its depth is <= znear, det <= 0 or its rectangle is empty.
 *   g: Gaussian SoA; count = counts->n_gaussians if counts != NULL else n_gauss
 *   means_relative: 1 if means are camera-relative (as written by ogs_decode), 0 if world
 *   rec ogs_rec2d[G], depth_key u32[G] (float bits of depth), rect u32[G][2]
 *   (x0 | y0 << 16, x1 | y1 << 16), tiles u32[G] (number of tiles covered)
 *   tile_count u32[grid_x * grid_y] (optional, may be NULL): zeroed by the call, then the
 *   number of (tile, Gaussian) pairs of every tile — pass it to ogs_sort, which then skips
 *   its own counting pass
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_project_bin(const ogs_gaussians* g /* host struct */, int64_t n_gauss,
                           int32_t means_relative, const ogs_camera* cam /* host */,
                           ogs_rec2d* rec, uint32_t* depth_key, uint32_t* rect,
                           uint32_t* tiles, uint32_t* tile_count, ogs_counts* counts,
                           void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_decode_project_bf16 — Sec. 3.2 (Eq. offsets, Eq. mlp) fused with Sec. 3.1 (Eq. 1 and
 * the EWA projection): the Gaussians decoded on the tensor cores are projected in the same
 * kernel, without passing through global memory.  The outputs are bit-for-bit those of
 * ogs_decode_bf16 (into `out`) followed by ogs_project_bin(out, sel_cap * k,
 * means_relative = 1, cam, rec, depth_key, rect, tiles, tile_count, counts).
 *   pos, feat, offs, lv, N, mlp, cam, sel_idx, sel_w, sel_cap, counts: as ogs_decode_bf16
 *   out (optional, may be NULL): the Gaussian SoA is also written (training needs it for the
 *   backward); NULL writes records only
 *   rec, depth_key, rect, tiles, tile_count (optional): as ogs_project_bin, counted over
 *   counts->n_gaussians Gaussians; tile_count is zeroed by the call
 *   scratch: ogs_decode_project_scratch_bytes() bytes, 16-byte aligned (the BF16 operand
 *   image of the decoder, packed by the call)
 * counts->timeout is set if a bounded internal wait expires (records of the remaining
 * anchors not written).
 * ------------------------------------------------------------------------------------- */
size_t ogs_decode_project_scratch_bytes(void);
ogs_status ogs_decode_project_bf16(const float* pos, const float* feat, const float* offs,
                                   const float* lv, int64_t N, const ogs_mlp* mlp /* host */,
                                   const ogs_camera* cam /* host */, const uint32_t* sel_idx,
                                   const float* sel_w, int64_t sel_cap, ogs_counts* counts,
                                   const ogs_gaussians* out /* host struct or NULL */,
                                   ogs_rec2d* rec, uint32_t* depth_key, uint32_t* rect,
                                   uint32_t* tiles, uint32_t* tile_count, void* scratch,
                                   size_t scratch_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_sort — Sec. 3.1: for every tile, the Gaussians whose rectangle covers it, in
 * front-to-back order (ascending depth, ties by Gaussian id).  Built per tile: pair counts per
 * tile and their exclusive scan (the tile ranges), an unordered fill of each tile's range, and
 * a sort of every range by the unique key (depth bits << 32 | Gaussian id) in shared memory
 * (one small CTA per list of up to 2048 pairs, larger CTAs for the few longer lists).  The
 * result is fully determined by the inputs.
 *   depth_key/rect/tiles from ogs_project_bin; tile_count (optional) the per-tile pair counts
 *   written by ogs_project_bin for the same Gaussians, or NULL to count here; n_gauss < 0
 *   takes the Gaussian count from
 *   counts->n_gaussians (as written by ogs_decode), else n_gauss (<= g_cap)
 *   pair_gauss u32[pair_cap]: Gaussian id of each pair, tile-major, front-to-back
 *   tile_range u32[n_tiles][2]: [start, end) of each tile in pair_gauss
 *   counts->n_pairs = P; if P > pair_cap, overflow bit 1 is set, need_pairs = P and no pair
 *   is emitted (every tile range is empty).
 *   scratch: ogs_sort_scratch_bytes(g_cap, pair_cap, n_tiles) bytes, 16-byte aligned.
 * ------------------------------------------------------------------------------------- */
size_t ogs_sort_scratch_bytes(int64_t g_cap, int64_t pair_cap, int32_t n_tiles);
ogs_status ogs_sort(const uint32_t* depth_key, const uint32_t* rect, const uint32_t* tiles,
                    const uint32_t* tile_count, int64_t g_cap, int64_t n_gauss,
                    int32_t grid_x, int32_t grid_y,
                    uint32_t* pair_gauss, uint32_t* tile_range, int64_t pair_cap,
                    ogs_counts* counts, void* scratch, size_t scratch_bytes, void* stream);

/* Per-tile pair regions: tile t owns the entries [t * tile_cap, t * tile_cap + count_t) of
 * pair_gauss (Gaussian id) and pair_key (its depth key).  Both arrays u32[n_tiles *
 * tile_cap], caller-owned. */
typedef struct ogs_tile_bins {
    uint32_t* pair_key;
    uint32_t* pair_gauss;
    uint32_t tile_cap;
} ogs_tile_bins;

/* ---------------------------------------------------------------------------------------
 * ogs_sort_bins — the tile lists of Sec. 3.1, as ogs_sort gives them (each tile's Gaussians
 * ordered by (depth key, id)), but each list in its tile's fixed region instead of packed:
 * one pass places every (Gaussian, tile) pair in its tile's region at the slot the atomic
 * that counts it returns, then every region is sorted in place.  No prefix scan and no
 * second pass over the pairs.  Rectangles of more than 8 tiles are handed on in chunks of
 * 1024 tiles to a second pass whose warps share them out over the grid (the scratch holds
 * 32 chunk entries per tile, at least 4096; chunks beyond that are placed by the first pass).
 *   depth_key, rect, tiles, g_cap, n_gauss, grid_x, grid_y: as ogs_sort
 *   bins: the regions (host struct); pair_gauss holds the sorted lists afterwards and
 *   pair_key is clobbered
 *   tile_range u32[n_tiles][2]: [t * tile_cap, t * tile_cap + count_t) of each tile
 *   counts->n_pairs = the number of pairs.  If a tile has more than tile_cap pairs, overflow
 *   bit 1 is set, need_pairs = the largest count (the tile_cap that fits) and every range is
 *   empty.
 *   scratch: ogs_sort_bins_scratch_bytes(n_tiles) bytes, 16-byte aligned.
 * ------------------------------------------------------------------------------------- */
size_t ogs_sort_bins_scratch_bytes(int32_t n_tiles);
ogs_status ogs_sort_bins(const uint32_t* depth_key, const uint32_t* rect, const uint32_t* tiles,
                         int64_t g_cap, int64_t n_gauss, int32_t grid_x, int32_t grid_y,
                         const ogs_tile_bins* bins /* host struct */, uint32_t* tile_range,
                         ogs_counts* counts, void* scratch, size_t scratch_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_radix_sort_pairs — a stable LSD radix sort of (key, value) pairs (the sort of the
 * cited rasterizer's global (tile, depth) key design; ogs_sort builds the same lists per tile
 * instead): sorts by bits [bit_lo, bit_hi) of the key, equal keys keeping their input
 * order.  n = *n_dev if n_dev != NULL (device count, <= n_cap) else n_cap.  Result
 * replaces keys/vals in place.
 *   scratch: ogs_radix_sort_scratch_bytes(n_cap) bytes, 16-byte aligned.
 * ------------------------------------------------------------------------------------- */
size_t ogs_radix_sort_scratch_bytes(int64_t n_cap);
ogs_status ogs_radix_sort_pairs(uint32_t* keys, uint32_t* vals, const uint32_t* n_dev,
                                int64_t n_cap, int32_t bit_lo, int32_t bit_hi, void* scratch,
                                size_t scratch_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_blend_fwd — Sec. 3.1, Eq. 2: per pixel, over its tile's list front to back:
 * alpha = min(0.99, o exp(power)); skip power > 0 or alpha < 1/255; stop before a Gaussian
 * that would bring T below 1e-4; C += c alpha T; T *= 1 - alpha.  Finally C += T bg.
 *   rec, pair_gauss, tile_range from the calls above
 *   bg: host float[3]
 *   img f32[3][H][W], T_final f32[H][W], n_last u32[H][W] (list entries up to and
 *   including the last blended one; optional, may be NULL when no backward follows: the
 *   kernel then skips tracking it); img may be pinned host memory (page-locked, so its
 *   address is valid on the device under unified addressing): the image then goes to the
 *   host while the kernel runs, with no separate copy
 *   n_eval (optional, may be NULL): u32[H][W], (pixel, Gaussian) tests the kernel made for
 *   the pixel while it still needed them: the list entries whose alpha >= 1/255 ellipse box
 *   reaches the pixel's 8x8 block, up to and including the one the pixel saturated on (the
 *   blend's unit of work as executed; entries whose box misses the block are never tested)
 *   maxc (optional, may be NULL): u32[N_anchors], float bits of the largest T*alpha of any
 *   blended Gaussian of each anchor (atomic max; caller zeroes); anchor of Gaussian g is
 *   sel_idx[g / k].
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_blend_fwd(const ogs_rec2d* rec, const uint32_t* pair_gauss,
                         const uint32_t* tile_range, int32_t width, int32_t height,
                         const float* bg /* host float[3] */, float* img, float* T_final,
                         uint32_t* n_last, uint32_t* n_eval, const uint32_t* sel_idx, int32_t k,
                         uint32_t* maxc, void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_blend_bwd — backward of ogs_blend_fwd (Sec. 3.1, Eq. 2).  With C = sum_i c_i a_i T_i +
 * T_{n+1} bg: dC/dc_i = a_i T_i, dC/da_i = T_i (c_i - S_i) with S the colour behind i.  Each
 * pixel replays its list back to front from n_last, recovering T_i = T_{i+1}/(1 - a_i) from
 * T_final (no per-pair storage); a = min(0.99, o G) has zero derivative where clamped.
 *   rec, pair_gauss, tile_range, T_final, n_last: as produced by the forward
 *   bg: host float[3];  dimg f32[3][H][W] = dL/dimage
 *   drec f32[G][9] (ACCUMULATED, caller zeroes): dL/d(u, v, conic a, conic b, conic c,
 *   opacity, r, g, b) per Gaussian.  Atomic accumulation: float summation order varies.
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_blend_bwd(const ogs_rec2d* rec, const uint32_t* pair_gauss,
                         const uint32_t* tile_range, int32_t width, int32_t height,
                         const float* bg /* host float[3] */, const float* T_final,
                         const uint32_t* n_last, const float* dimg, float* drec, void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_project_bwd — backward of the EWA projection of ogs_project_bin (Sec. 3.1, Eq. 1):
 * d(u, v, conic) -> d(mean, scale, unit quaternion).  Gaussians with an empty rect get 0.
 *   g, means_relative, cam: as given to ogs_project_bin; rect from it; drec from
 *   ogs_blend_bwd; count = counts->n_gaussians if counts != NULL else n_gauss
 *   dmeans f32[G][3], dscales f32[G][3], dquats f32[G][4] (written, not accumulated)
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_project_bwd(const ogs_gaussians* g /* host struct */, int64_t n_gauss,
                           int32_t means_relative, const ogs_camera* cam /* host */,
                           const uint32_t* rect, const float* drec, float* dmeans,
                           float* dscales, float* dquats, const ogs_counts* counts,
                           void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_decode_bwd — backward of ogs_decode (Sec. 3.2, Eq. offsets and Eq. mlp): per selected
 * anchor, recomputes the three decoders and chains the per-Gaussian gradients (dmeans,
 * dscales, dquats from ogs_project_bwd; opacity and colour gradients from drec) into
 *   dfeat f32[N][F], doffs f32[N][k][3], dlv f32[N][3]   (ACCUMULATED: +=)
 *   dmlp: decoder weight gradients, same layout as ogs_mlp  (ACCUMULATED: +=); with
 *   appearance codes (mlp->A > 0) also dmlp->w1_app f32[H][A] and the code gradients
 *   dmlp->app f32[N][A] (both +=, both required; dmlp->A is ignored)
 * Anchor positions, LOD bias and the selection are constants.  A row pass (thread per
 * anchor) writes each anchor's output, hidden and input rows to scratch; weight gradients are
 * summed per block over those rows and then across blocks in a fixed order (deterministic).
 *   sel_idx/sel_w: the selection the forward decoded (counts->n_selected <= sel_cap entries)
 *   feat and dfeat 16-byte aligned
 *   scratch: ogs_decode_bwd_scratch_bytes(sel_cap) bytes, 16-byte aligned (about 1.4 KB per
 *   selectable anchor plus 8.7 MB).
 * ------------------------------------------------------------------------------------- */
size_t ogs_decode_bwd_scratch_bytes(int64_t sel_cap);
ogs_status ogs_decode_bwd(const float* pos, const float* feat, const float* offs, const float* lv,
                          int64_t N, const ogs_mlp* mlp /* host struct */,
                          const ogs_camera* cam /* host */, const uint32_t* sel_idx,
                          const float* sel_w, int64_t sel_cap, const ogs_counts* counts,
                          const float* dmeans,
                          const float* dscales, const float* dquats, const float* drec,
                          float* dfeat, float* doffs, float* dlv,
                          const ogs_mlp* dmlp /* host struct of device ptrs, written */,
                          void* scratch, size_t scratch_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_decode_bwd_bf16 — ogs_decode_bwd with the per-anchor products on the tensor cores
 * (tcgen05, BF16 operands, FP32 accumulation in tensor memory): the recomputed decoder
 * layers, dy . W2 and dp . W1 take BF16-rounded inputs, weights and gradients (relative
 * 2^-9 each); the output gradients dy, the ReLU masks, the weight-gradient products over the
 * anchors and every accumulation stay FP32.  The backward of ogs_decode_bf16.  Same
 * arguments, scratch and results as ogs_decode_bwd, except that counts is written: on a
 * tensor-core wait that does not complete, counts->timeout is set.  Appearance codes enter
 * the recomputed first layer as BF16 K columns 40..47; their gradients (dmlp->app, w1_app)
 * are formed in FP32 from the FP32 pre-activation gradients.
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_decode_bwd_bf16(const float* pos, const float* feat, const float* offs,
                               const float* lv, int64_t N, const ogs_mlp* mlp /* host struct */,
                               const ogs_camera* cam /* host */, const uint32_t* sel_idx,
                               const float* sel_w, int64_t sel_cap, ogs_counts* counts,
                               const float* dmeans, const float* dscales, const float* dquats,
                               const float* drec, float* dfeat, float* doffs, float* dlv,
                               const ogs_mlp* dmlp /* host struct of device ptrs, written */,
                               void* scratch, size_t scratch_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_loss_l1 — photometric L1 term of Sec. 5.1.5: loss = mean |img - target| over n
 * values; dimg = sign(img - target) / n (written); *loss += the mean (device float, caller
 * zeroes; may be NULL).
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_loss_l1(const float* img, const float* target, int64_t n, float* dimg,
                       float* loss, void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_loss_l1_ssim — photometric loss of Sec. 5.1.5: (1 - lambda) L1 + lambda (1 - SSIM)
 * (lambda = 0.2 in the paper), SSIM with an 11x11 Gaussian window (sigma 1.5, zero padded),
 * C1 = 0.01^2, C2 = 0.03^2, averaged over the C x H x W values.  dimg (written) is the
 * gradient w.r.t. img; *loss += the loss (device float, may be NULL).
 *   target_stats (optional, may be NULL): f32[2][C][H][W], the target's window moments G*y
 *   and G*y^2 as written by ogs_ssim_target_stats for this target; with them the forward pass
 *   blurs three moments instead of five (same loss and gradient up to FP32 rounding).
 *   scratch: ogs_loss_l1_ssim_scratch_bytes(C, H, W) bytes, 16-byte aligned.
 * ogs_ssim_target_stats — the two window moments of a target image (zero padded), for reuse
 * by every loss evaluation against that target.
 * ------------------------------------------------------------------------------------- */
size_t ogs_loss_l1_ssim_scratch_bytes(int32_t C, int32_t H, int32_t W);
ogs_status ogs_loss_l1_ssim(const float* img, const float* target, int32_t C, int32_t H,
                            int32_t W, float lambda, float* dimg, float* loss,
                            const float* target_stats, void* scratch, size_t scratch_bytes,
                            void* stream);
ogs_status ogs_ssim_target_stats(const float* target, int32_t C, int32_t H, int32_t W,
                                 float* target_stats, void* stream);

/* ---------------------------------------------------------------------------------------
 * Adam over touched anchor rows (the optimiser step of the training loop, Sec. 5.1.5, over
 * the anchors a step's views selected).  Anchors outside every view of a step receive no
 * gradient; their parameters and moments are left as they are (lazy Adam: a row's moments
 * decay only on the steps that touch it, bias correction uses the global step count), so a
 * step streams only the touched rows instead of every anchor's state.
 *
 * ogs_stamp_selected — stamp[sel_idx[r]] = value for r < counts->n_selected (call once per
 *   view of the step with value = the step number; stamp u32[N], caller-owned, zeroed once).
 * ogs_adam_rows — for every row j < rows with stamp[j] == value, one Adam update of its
 *   row_len values (param/grad/m/v f32[rows][row_len]) as ogs_adam (same bias correction with
 *   the 1-based global `step`); zero_grad != 0 clears the updated rows' gradients.  Rows with
 *   another stamp are not read or written beyond their stamp.
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_stamp_selected(const uint32_t* sel_idx, const ogs_counts* counts,
                              int64_t sel_cap, uint32_t* stamp, uint32_t value, void* stream);
ogs_status ogs_adam_rows(float* param, float* grad, float* m, float* v, int64_t rows,
                         int32_t row_len, const uint32_t* stamp, uint32_t value, float lr,
                         float beta1, float beta2, float eps, int32_t step, int32_t zero_grad,
                         void* stream);

/* ---------------------------------------------------------------------------------------
 * Error surface.  The library keeps no context: a frame's device-side error state is its
 * ogs_counts record (overflow bits, timeout) plus, on request, a non-finite flag word.
 *
 * ogs_scan_nonfinite — opt-in check of any f32 buffer (inputs, images, gradients): *flag |= bit
 *   (device u32, caller zeroes) if any of x[0..n) is NaN or infinite.  Enqueued like every
 *   call; nothing is synchronised.
 * ogs_counts_status — host function: maps a copy of ogs_counts (read back by the caller) and a
 *   non-finite flag word to a status: OGS_ERR_NONFINITE if the flag is set, else
 *   OGS_ERR_TIMEOUT if a bounded wait expired, else OGS_ERR_CAPACITY if a capacity
 *   overflowed (the needed sizes are in the record), else OGS_OK.
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_scan_nonfinite(const float* x, int64_t n, uint32_t* flag, uint32_t bit,
                              void* stream);
ogs_status ogs_counts_status(const ogs_counts* counts /* host */, uint32_t nonfinite);

/* ---------------------------------------------------------------------------------------
 * ogs_scale — x[i] *= *s for i < n (s a device float).  The backward of a loss that enters a
 * larger objective multiplies the loss's own gradient (dimg of ogs_loss_l1 /
 * ogs_loss_l1_ssim) by the gradient arriving from that objective (the chain rule of the
 * autograd wrappers); reading s on the device needs no host synchronisation.
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_scale(float* x, int64_t n, const float* s, void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_adam — one Adam step over n parameters (step >= 1 is the 1-based step count used for
 * bias correction):  m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).  zero_grad != 0 clears g.
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_adam(float* param, float* grad, float* m, float* v, int64_t n, float lr,
                    float beta1, float beta2, float eps, int32_t step, int32_t zero_grad,
                    void* stream);

/* ---------------------------------------------------------------------------------------
 * ogs_radix_sort_pairs_noalloc — the same stable LSD radix sort as ogs_radix_sort_pairs, for
 * callers that cannot allocate device memory (an embedding host application that owns the
 * device heap and offers no allocator, or a real-time frame loop that must not call
 * cudaMalloc/cudaFree because they synchronise the device).  The paper has no counterpart:
 * this is a deployment variant of the sort.
 *   Scratch is a fixed array inside the library image (about 9.4 MB), reserved on every GPU
 *   that loads the library until the process exits; no allocation of any kind is made.
 *   n_cap must be <= ogs_radix_sort_pairs_noalloc_max_items() (2^20); larger requests return
 *   OGS_ERR_CAPACITY and enqueue nothing.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *   which may load the module): make that first call before any stream capture.
 *   All calls share the one array, so calls that overlap on the GPU (different streams
 *   without ordering, or different host threads) race; serialise them.  The array keeps the
 *   last call's contents; every word is written before it is read, so nothing is cleared.
 *   Other arguments and the result are as for ogs_radix_sort_pairs.
 * ------------------------------------------------------------------------------------- */
int64_t ogs_radix_sort_pairs_noalloc_max_items(void);
ogs_status ogs_radix_sort_pairs_noalloc(uint32_t* keys, uint32_t* vals, const uint32_t* n_dev,
                                        int64_t n_cap, int32_t bit_lo, int32_t bit_hi,
                                        void* stream);

/* ---------------------------------------------------------------------------------------
 * Explicit Gaussians per anchor ("Our-3D-GS", Sec. 5): each anchor carries k explicit 3D
 * Gaussians (per-Gaussian SoA, anchor-major: element [j][i] of anchor j, slot i):
 *   log_scale f32[N][k][3], quat f32[N][k][4] (w, x, y, z; 16-byte aligned), opacity
 *   f32[N][k] (logits), color_dc f32[N][k][3] (degree-0 spherical-harmonic coefficients)
 * ------------------------------------------------------------------------------------- */
typedef struct ogs_explicit {
    const float* log_scale;
    const float* quat;
    const float* opacity;
    const float* color_dc;
} ogs_explicit;

/* ogs_explicit_gaussians — in place of ogs_decode: for every selected anchor j (weight w) and
 * slot i, mean x_j - campos + O_ji * l_j (Eq. offsets, camera-relative like ogs_decode),
 * scale exp(log_scale), unit quaternion, opacity w sigmoid(opacity), colour
 * max(0, 0.28209479 color_dc + 1/2) (the cited 3D-GS activations).  Reads M from
 * counts->n_selected; writes Gaussians 0 .. M*k-1 of out (same layout as ogs_decode). */
ogs_status ogs_explicit_gaussians(const float* pos, const float* offs, const float* lv,
                                  int64_t N, int32_t k, const ogs_explicit* attr /* host */,
                                  const ogs_camera* cam /* host */, const uint32_t* sel_idx,
                                  const float* sel_w, int64_t sel_cap, const ogs_counts* counts,
                                  const ogs_gaussians* out /* host struct */, void* stream);

/* ogs_explicit_gaussians_bwd — backward of ogs_explicit_gaussians: per-Gaussian dmeans,
 * dscales, dquats (ogs_project_bwd) and the opacity / colour gradients of drec
 * (ogs_blend_bwd) into grad (same layout as attr, ACCUMULATED), doffs f32[N][k][3] and
 * dlv f32[N][3] (ACCUMULATED). */
ogs_status ogs_explicit_gaussians_bwd(const float* pos, const float* offs, const float* lv,
                                      int64_t N, int32_t k, const ogs_explicit* attr /* host */,
                                      const ogs_camera* cam /* host */, const uint32_t* sel_idx,
                                      const float* sel_w, int64_t sel_cap,
                                      const ogs_counts* counts, const float* dmeans,
                                      const float* dscales, const float* dquats,
                                      const float* drec, const ogs_explicit* grad /* host */,
                                      float* doffs, float* dlv, void* stream);

/* ---------------------------------------------------------------------------------------
 * View-frequency anchor pruning (Sec. 4.2.2): anchors whose view frequency (fraction of the
 * training views that select them) is below tau_v are removed.
 *   ogs_count_selected: sel_count[j] += 1 for the counts->n_selected entries of sel_idx
 *   (one view's selection; an anchor appears at most once per view).
 *   ogs_prune_anchors: keep_idx u32[N] receives, in ascending order, the anchors with
 *   sel_count >= min_count, and *n_kept (device) their number.  min_count is the smallest
 *   count whose frequency count / n_views is not below tau_v (computed by the caller).
 *   scratch: ogs_prune_scratch_bytes(N) bytes, 16-byte aligned.
 *   ogs_gather_rows: dst row r = src row keep_idx[r] for r < min(*n_dev, n_cap) (n_dev may
 *   be NULL: n_cap rows); rows of row_bytes bytes (any per-anchor array); src != dst.
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_count_selected(const uint32_t* sel_idx, const ogs_counts* counts,
                              uint32_t* sel_count, void* stream);
size_t ogs_prune_scratch_bytes(int64_t N);
ogs_status ogs_prune_anchors(const uint32_t* sel_count, int64_t N, uint32_t min_count,
                             uint32_t* keep_idx, uint32_t* n_kept, void* scratch,
                             size_t scratch_bytes, void* stream);
ogs_status ogs_gather_rows(const void* src, void* dst, int64_t row_bytes, const uint32_t* idx,
                           const uint32_t* n_dev, int64_t n_cap, void* stream);

/* ---------------------------------------------------------------------------------------
 * Average-opacity anchor pruning (Sec. 4.2.2): anchors whose Gaussians' average opacity over
 * the counted training views is below tau_o are removed.
 *   ogs_opacity_accumulate: for the counts->n_selected anchors of one view's selection,
 *   opac_sum[sel_idx[r]] += sum_i max(opac[r k + i], 0) (FP32, slots in order; opac as
 *   written by the decoder, f32[G]) and opac_views[sel_idx[r]] += 1.  opac_sum f32[N],
 *   opac_views u32[N] (caller zeroes).
 *   ogs_prune_by_opacity: keep_idx u32[N] receives, in ascending order, every anchor except
 *   those with opac_views > 0 and opac_sum / (opac_views k) < tau_o (FP32 quotient);
 *   *n_kept (device) their number.  scratch: ogs_prune_opacity_scratch_bytes(N) bytes,
 *   16-byte aligned.  Compact the per-anchor arrays with ogs_gather_rows.
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_opacity_accumulate(const float* opac, const uint32_t* sel_idx,
                                  const ogs_counts* counts, int32_t k, float* opac_sum,
                                  uint32_t* opac_views, void* stream);
size_t ogs_prune_opacity_scratch_bytes(int64_t N);
ogs_status ogs_prune_by_opacity(const float* opac_sum, const uint32_t* opac_views, int64_t N,
                                int32_t k, float tau_o, uint32_t* keep_idx, uint32_t* n_kept,
                                void* scratch, size_t scratch_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * Learned anchor-visibility proposal (not in the paper: a gate in front of decoding).  A
 * 3-layer MLP, input x = [f_v (32), L/(NL-1), unit viewing direction in the camera frame
 * R (x_v - campos)/d (3), ln(d/d_max)] (37), hidden 64 ReLU, 64 ReLU, output keep probability
 * p = sigmoid(w3 . h2 + b3).
 *   w1 f32[64][37], b1 f32[64], w2 f32[64][64], b2 f32[64], w3 f32[64], b3 f32[1]
 * ------------------------------------------------------------------------------------- */
typedef struct ogs_proposal {
    const float* w1;
    const float* b1;
    const float* w2;
    const float* b2;
    const float* w3;
    const float* b3;
} ogs_proposal;

/* ogs_proposal_gate — scores the counts->n_selected entries of (sel_in, w_in) and writes the
 * ones with p >= p_star to (sel_out, w_out) in their original order; counts->n_selected and
 * n_gaussians are updated to the kept count.  p_out (optional) receives p for every input
 * entry.  sel_out must not alias sel_in.
 *   scratch: ogs_proposal_gate_scratch_bytes(sel_cap) bytes, 16-byte aligned. */
size_t ogs_proposal_gate_scratch_bytes(int64_t sel_cap);
ogs_status ogs_proposal_gate(const float* pos, const uint8_t* level, const float* feat,
                             int64_t N, int32_t NL, int32_t k, const ogs_camera* cam /* host */,
                             const ogs_proposal* net /* host struct */, float p_star,
                             const uint32_t* sel_in, const float* w_in, int64_t sel_cap,
                             ogs_counts* counts, uint32_t* sel_out, float* w_out, float* p_out,
                             void* scratch, size_t scratch_bytes, void* stream);

/* ogs_proposal_gate_bf16 — ogs_proposal_gate with both hidden layers computed as BF16 x BF16
 * -> FP32 tensor-core products (inputs and first hidden layer rounded to BF16; biases, ReLU,
 * the output layer and the sigmoid in FP32).  Same arguments, scratch and results; p differs
 * from the FP32 form by the BF16 rounding, so entries with p near p_star may be decided
 * differently.  On a tensor-core wait that does not complete, counts->timeout is set. */
ogs_status ogs_proposal_gate_bf16(const float* pos, const uint8_t* level, const float* feat,
                                  int64_t N, int32_t NL, int32_t k,
                                  const ogs_camera* cam /* host */,
                                  const ogs_proposal* net /* host struct */, float p_star,
                                  const uint32_t* sel_in, const float* w_in, int64_t sel_cap,
                                  ogs_counts* counts, uint32_t* sel_out, float* w_out,
                                  float* p_out, void* scratch, size_t scratch_bytes,
                                  void* stream);

/* ogs_lod_select_gated — ogs_lod_select followed by ogs_proposal_gate_bf16, in one pass over
 * the anchors: inside the selection's tile pass, the anchors kept by the LOD rule are scored by
 * the same tensor-core network arithmetic as ogs_proposal_gate_bf16 (so every keep decision is
 * the same), and only the anchors that pass both are listed, in ascending order, with their
 * LOD weights.  sel_idx, sel_w, counts->n_selected and n_gaussians are those of the two calls
 * whenever neither overflows; here the capacity check (sel_cap, overflow bit 0, need_selected)
 * applies to the gated list.  No keep probabilities are returned.
 *   pos, level, dL, N, NL, k, cam, infer: as ogs_lod_select; feat f32[N][32] (16-byte
 *   aligned), net, p_star: as ogs_proposal_gate_bf16
 *   scratch: ogs_lod_select_gated_scratch_bytes(N) bytes, 16-byte aligned.
 *   counts: every field is reset to zero by the call before anything else writes it (the
 *   start of a frame's counters; the caller need not clear them).
 * On a tensor-core wait that does not complete, counts->timeout is set (that tile's anchors
 * keep their LOD selection). */
size_t ogs_lod_select_gated_scratch_bytes(int64_t N);
ogs_status ogs_lod_select_gated(const float* pos, const uint8_t* level, const float* dL,
                                const float* feat, int64_t N, int32_t NL, int32_t k,
                                const ogs_camera* cam /* host */, int32_t infer,
                                const ogs_proposal* net /* host struct */, float p_star,
                                uint32_t* sel_idx, float* sel_w, int64_t sel_cap,
                                ogs_counts* counts, void* scratch, size_t scratch_bytes,
                                void* stream);

/* ogs_proposal_train — mean weighted binary cross-entropy of the keep probability over the
 * selected anchors of one view against labels y = (maxc[anchor] >= tau) (maxc as written by
 * ogs_blend_fwd: float bits of the largest T*alpha), positives weighted by pos_weight (> 0),
 * and its gradients.
 *   grads: same layout as the network, ACCUMULATED (+=); *loss += mean BCE (may be NULL).
 *   dloss: device float (may be NULL, meaning 1), the gradient of the caller's objective with
 *   respect to this BCE; every gradient added to grads is multiplied by it (the backward of a
 *   loss that enters a larger objective).
 *   scratch: ogs_proposal_train_scratch_bytes() bytes, 16-byte aligned. */
size_t ogs_proposal_train_scratch_bytes(void);
ogs_status ogs_proposal_train(const float* pos, const uint8_t* level, const float* feat,
                              int64_t N, int32_t NL, const ogs_camera* cam /* host */,
                              const ogs_proposal* net /* host struct */, const uint32_t* sel_idx,
                              const ogs_counts* counts, const uint32_t* maxc, float tau,
                              float pos_weight,
                              const ogs_proposal* grads /* host struct, written */, float* loss,
                              const float* dloss, void* scratch, size_t scratch_bytes,
                              void* stream);

/* ---------------------------------------------------------------------------------------
 * Anchor growing and the LOD-bias update (Sec. 4.2.1).  Over the training views between two
 * densification steps, every neural Gaussian (anchor j, slot i) accumulates the norm of its
 * view-space position gradient; the average over the views that saw it, grad_g, decides:
 *   - growing: with tau[L] = tau_g * 2^(beta L) (per level, FP32, given by the caller), a
 *     Gaussian of an anchor of level L with grad_g > tau[L + 1] (and L + 1 < NL) proposes a
 *     new anchor at level L + 1 ("next level"), else with grad_g > tau[L] one at level L.
 *     The proposal is the voxel of the target level L' holding the Gaussian's position
 *     mu = pos_j + offs_ji * l_v (FP32: product, then sum); voxels are centred on the grid
 *     points of spacing voxel[L'] = delta / 2^L' (given), as in the Eq. for V_L, so the
 *     voxel index is rint(mu / voxel[L']) per axis (FP32 quotient, ties to even).  It
 *     becomes an anchor only if no anchor of that level lies in that voxel (an anchor's own
 *     voxel: rint(pos / voxel) at its level), and among proposals of the same new voxel the
 *     one with the smallest index j k + i wins.  New anchors sit at the voxel centre, the
 *     grid point index * voxel[L'].
 *   - LOD bias: grad_v = (sum_i acc_ji) / (sum_i cnt_ji) (FP32, slots summed in order); an
 *     anchor of level L with grad_v > thr_bias[L] (the caller passes 0.25 tau[L]) gets
 *     dL += eps.
 * Voxel coordinates must lie in [-2^19, 2^19) per axis and NL <= 15; an anchor or proposal
 * outside that range takes no part in growing.
 *
 *   ogs_grow_accumulate: for each Gaussian g < counts->n_gaussians of one view with
 *   tiles[g] > 0 (its projection touches a tile): grad_acc[j][i] += |(du W/2, dv H/2)|
 *   (drec columns 0 and 1, the pixel-space mean gradient, scaled to normalised device
 *   coordinates) and grad_cnt[j][i] += 1, where j = sel_idx[g / k], i = g % k.  An anchor
 *   appears once per view, so the call needs no atomics; drec, tiles: as from ogs_blend_bwd
 *   and ogs_project_bin / ogs_decode_project_bf16.  grad_acc f32[N][k], grad_cnt u32[N][k]
 *   (the caller zeroes them after each densification step).
 *   ogs_update_lod_bias: dL[j] += eps where grad_v > thr_bias[level_j] (host float[NL]).
 *   ogs_grow_anchors: the proposals above, written as new anchor rows r < n_new[0]:
 *   new_pos f32[max_new][3] (voxel centre), new_level u8[max_new], new_lv f32[max_new][3]
 *   (the voxel size on every axis), parent u32[max_new] (the proposing anchor, whose other
 *   attributes the caller copies, e.g. with ogs_gather_rows), in increasing j k + i.
 *   n_new u32[2] (device): [0] rows written = min(needed, max_new), [1] rows needed; the
 *   call is deterministic, so a caller that finds [1] > max_new grows the buffers and calls
 *   again.  tau, voxel: host float[NL].  next_level = 0 disables the promotion to L + 1
 *   (proposals at the Gaussian's own level only: the progressive stage of Sec. 4.3).  N k < 2^32 - 1; with N = 0 the anchor arrays may be NULL.
 *   scratch: ogs_grow_scratch_bytes(N, k) bytes, 16-byte aligned (a hash table of 2^ceil(
 *   log2(2 N (k + 1))) voxel keys at 12 bytes each, plus 12 bytes per proposal slot).
 * ------------------------------------------------------------------------------------- */
ogs_status ogs_grow_accumulate(const float* drec, const uint32_t* tiles, const uint32_t* sel_idx,
                               const ogs_counts* counts, int32_t k, int32_t width,
                               int32_t height, float* grad_acc, uint32_t* grad_cnt,
                               void* stream);
ogs_status ogs_update_lod_bias(const uint8_t* level, const float* grad_acc,
                               const uint32_t* grad_cnt, int64_t N, int32_t k, int32_t NL,
                               const float* thr_bias /* host float[NL] */, float eps, float* dL,
                               void* stream);
size_t ogs_grow_scratch_bytes(int64_t N, int32_t k);
ogs_status ogs_grow_anchors(const float* pos, const uint8_t* level, const float* offs,
                            const float* lv, const float* grad_acc, const uint32_t* grad_cnt,
                            int64_t N, int32_t k, int32_t NL,
                            const float* tau /* host float[NL] */,
                            const float* voxel /* host float[NL] */, int32_t next_level,
                            float* new_pos,
                            uint8_t* new_level, float* new_lv, uint32_t* parent,
                            int64_t max_new, uint32_t* n_new, void* scratch,
                            size_t scratch_bytes, void* stream);

/* Library version string (host). */
const char* ogs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OGS_H */
