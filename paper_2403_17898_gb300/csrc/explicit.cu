// Explicit Gaussians per anchor (the "Our-3D-GS" variant of Sec. 5: each anchor carries k
// explicit 3D Gaussians instead of decoding neural ones).  Positions follow Eq. offsets
// (x_v + O_i * l_v, written camera-relative like ogs_decode), the other attributes take the
// activations of the cited 3D-GS: scale exp(s), unit quaternion, opacity sigmoid(a) times the
// anchor's LOD weight, colour max(0, SH_C0 f + 1/2) from the degree-0 harmonic.  The rest of
// the path (projection, lists, blending and their backward) is shared with the neural form.
//
// One thread per (selected anchor, Gaussian); HBM-bound gathers and streaming writes.
#include "internal.cuh"

namespace ogs {
namespace {

constexpr int kExThreads = 256;
constexpr float kShC0 = 0.28209479177387814f;

struct ExArgs {
    const float* pos;
    const float* offs;
    const float* lv;
    ogs_explicit attr;
    const uint32_t* sel_idx;
    const float* sel_w;
    const ogs_counts* counts;
    int k;
    Cam cam;
};

__global__ void __launch_bounds__(kExThreads) explicit_fwd(ExArgs a, ogs_gaussians out) {
    const uint32_t M = a.counts->n_selected;
    const uint64_t G = (uint64_t)M * a.k;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(g / a.k), i = (uint32_t)(g % a.k);
        const uint32_t j = a.sel_idx[r];
        const float w = a.sel_w[r];
        const size_t ji = (size_t)j * a.k + i;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float l = a.lv[3 * (size_t)j + q];
            out.means[3 * g + q] = (a.pos[3 * (size_t)j + q] - a.cam.c[q]) + a.offs[3 * ji + q] * l;
            out.scales[3 * g + q] = expf(a.attr.log_scale[3 * ji + q]);
            out.colors[3 * g + q] = fmaxf(fmaf(kShC0, a.attr.color_dc[3 * ji + q], 0.5f), 0.0f);
        }
        const float4 qv = *reinterpret_cast<const float4*>(a.attr.quat + 4 * ji);
        const float inv = 1.0f / sqrtf(qv.x * qv.x + qv.y * qv.y + qv.z * qv.z + qv.w * qv.w);
        *reinterpret_cast<float4*>(out.quats + 4 * g) =
            make_float4(qv.x * inv, qv.y * inv, qv.z * inv, qv.w * inv);
        out.opac[g] = w / (1.0f + expf(-a.attr.opacity[ji]));
    }
}

// Backward: per-Gaussian gradients (dmeans, dscales, dquats from ogs_project_bwd; opacity and
// colour from the record gradients of ogs_blend_bwd) into the attributes.  A Gaussian of a
// view belongs to one (anchor, slot), so its attribute and offset gradients accumulate without
// atomics; the anchor's l_v gradient gathers its k Gaussians with atomic adds.
__global__ void __launch_bounds__(kExThreads) explicit_bwd(ExArgs a, const float* __restrict__ dmeans,
                                                           const float* __restrict__ dscales,
                                                           const float* __restrict__ dquats,
                                                           const float* __restrict__ drec,
                                                           ogs_explicit grad, float* doffs,
                                                           float* dlv) {
    const uint32_t M = a.counts->n_selected;
    const uint64_t G = (uint64_t)M * a.k;
    float* gls = const_cast<float*>(grad.log_scale);
    float* gq = const_cast<float*>(grad.quat);
    float* go = const_cast<float*>(grad.opacity);
    float* gc = const_cast<float*>(grad.color_dc);
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(g / a.k), i = (uint32_t)(g % a.k);
        const uint32_t j = a.sel_idx[r];
        const float w = a.sel_w[r];
        const size_t ji = (size_t)j * a.k + i;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float dm = dmeans[3 * g + q];
            doffs[3 * ji + q] += dm * a.lv[3 * (size_t)j + q];
            atomicAdd(dlv + 3 * (size_t)j + q, dm * a.offs[3 * ji + q]);
            gls[3 * ji + q] += dscales[3 * g + q] * expf(a.attr.log_scale[3 * ji + q]);
            const float f = a.attr.color_dc[3 * ji + q];
            gc[3 * ji + q] += fmaf(kShC0, f, 0.5f) > 0.0f ? drec[9 * g + 6 + q] * kShC0 : 0.0f;
        }
        const float4 qv = *reinterpret_cast<const float4*>(a.attr.quat + 4 * ji);
        const float4 gv = *reinterpret_cast<const float4*>(dquats + 4 * g);
        const float inv = 1.0f / sqrtf(qv.x * qv.x + qv.y * qv.y + qv.z * qv.z + qv.w * qv.w);
        const float qn[4] = {qv.x * inv, qv.y * inv, qv.z * inv, qv.w * inv};
        const float ga[4] = {gv.x, gv.y, gv.z, gv.w};
        const float dot = qn[0] * ga[0] + qn[1] * ga[1] + qn[2] * ga[2] + qn[3] * ga[3];
        float4 acc = *reinterpret_cast<float4*>(gq + 4 * ji);
        acc.x += (ga[0] - qn[0] * dot) * inv;
        acc.y += (ga[1] - qn[1] * dot) * inv;
        acc.z += (ga[2] - qn[2] * dot) * inv;
        acc.w += (ga[3] - qn[3] * dot) * inv;
        *reinterpret_cast<float4*>(gq + 4 * ji) = acc;
        const float sg = 1.0f / (1.0f + expf(-a.attr.opacity[ji]));
        go[ji] += drec[9 * g + 5] * w * sg * (1.0f - sg);
    }
}

bool attr_ok(const ogs_explicit* e) {
    return e && e->log_scale && e->quat && e->opacity && e->color_dc && aligned(e->quat, 16);
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" ogs_status ogs_explicit_gaussians(const float* pos, const float* offs, const float* lv,
                                             int64_t N, int32_t k, const ogs_explicit* attr,
                                             const ogs_camera* cam, const uint32_t* sel_idx,
                                             const float* sel_w, int64_t sel_cap,
                                             const ogs_counts* counts, const ogs_gaussians* out,
                                             void* stream) {
    if (!pos || !offs || !lv || !attr_ok(attr) || !cam || !sel_idx || !sel_w || !counts || !out)
        return OGS_ERR_ARG;
    if (N < 0 || k < 1 || sel_cap < 0) return OGS_ERR_ARG;
    if (!out->means || !out->scales || !out->quats || !out->opac || !out->colors ||
        !aligned(out->quats, 16))
        return OGS_ERR_ARG;
    if (sel_cap == 0) return OGS_OK;
    ExArgs a{pos, offs, lv, *attr, sel_idx, sel_w, counts, k, make_cam(*cam)};
    explicit_fwd<<<stride_grid(sel_cap * k, kExThreads, 8), kExThreads, 0, (cudaStream_t)stream>>>(
        a, *out);
    return launch_status();
}

extern "C" ogs_status ogs_explicit_gaussians_bwd(const float* pos, const float* offs,
                                                 const float* lv, int64_t N, int32_t k,
                                                 const ogs_explicit* attr,
                                                 const ogs_camera* cam, const uint32_t* sel_idx,
                                                 const float* sel_w, int64_t sel_cap,
                                                 const ogs_counts* counts, const float* dmeans,
                                                 const float* dscales, const float* dquats,
                                                 const float* drec, const ogs_explicit* grad,
                                                 float* doffs, float* dlv, void* stream) {
    if (!pos || !offs || !lv || !attr_ok(attr) || !cam || !sel_idx || !sel_w || !counts ||
        !dmeans || !dscales || !dquats || !drec || !attr_ok(grad) || !doffs || !dlv)
        return OGS_ERR_ARG;
    if (N < 0 || k < 1 || sel_cap < 0 || !aligned(dquats, 16)) return OGS_ERR_ARG;
    if (sel_cap == 0) return OGS_OK;
    ExArgs a{pos, offs, lv, *attr, sel_idx, sel_w, counts, k, make_cam(*cam)};
    explicit_bwd<<<stride_grid(sel_cap * k, kExThreads, 8), kExThreads, 0, (cudaStream_t)stream>>>(
        a, dmeans, dscales, dquats, drec, *grad, doffs, dlv);
    return launch_status();
}
