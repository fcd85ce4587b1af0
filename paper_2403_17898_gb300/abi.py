"""Thin Python binding of the C ABI in ``include/ogs.h`` (argument marshalling only).

Every function here has the name of its C entry point without the ``ogs_`` prefix, takes
CUDA tensors (device memory) plus plain numbers, and enqueues the call on the current torch
stream (or ``stream``).  All arithmetic happens in ``libogs.so``; if the library is missing
the import fails with an error instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libogs.so")

STATUS = {0: "OGS_OK", 1: "OGS_ERR_ARG", 2: "OGS_ERR_CAPACITY", 3: "OGS_ERR_TIMEOUT",
          4: "OGS_ERR_CUDA"}


class OgsError(RuntimeError):
    pass


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("campos", C.c_float * 3), ("fx", C.c_float),
                ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32), ("znear", C.c_float), ("d_max", C.c_float),
                ("s", C.c_float), ("pad", C.c_float)]


class Counts(C.Structure):
    _fields_ = [(n, C.c_uint32) for n in ("n_selected", "n_gaussians", "n_pairs", "overflow",
                                          "need_selected", "need_pairs", "timeout", "reserved")]


COUNT_FIELDS = [f[0] for f in Counts._fields_]


class MLP(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("w1", "b1", "w2_op", "b2_op", "w2_col", "b2_col",
                                          "w2_cov", "b2_cov")] + \
               [("F", C.c_int32), ("H", C.c_int32), ("k", C.c_int32), ("A", C.c_int32),
                ("w1_app", C.c_void_p), ("app", C.c_void_p)]


class Proposal(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("w1", "b1", "w2", "b2", "w3", "b3")]


class Gaussians(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("means", "scales", "quats", "opac", "colors")]


class TileBins(C.Structure):
    """ogs_tile_bins: per-tile pair regions (pair_key, pair_gauss u32[n_tiles * tile_cap])."""
    _fields_ = [("pair_key", C.c_void_p), ("pair_gauss", C.c_void_p), ("tile_cap", C.c_uint32)]


_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_SZ = C.c_size_t

class Explicit(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("log_scale", "quat", "opacity", "color_dc")]


_SIGS = {
    "ogs_lod_select_scratch_bytes": (_SZ, [_I64]),
    "ogs_lod_select": (C.c_int, [_P, _P, _P, _I64, _I32, _I32, C.POINTER(Camera), _I32, _P, _P,
                                 _I64, _P, _P, _SZ, _P]),
    "ogs_lod_select_gated_scratch_bytes": (_SZ, [_I64]),
    "ogs_lod_select_gated": (C.c_int, [_P, _P, _P, _P, _I64, _I32, _I32, C.POINTER(Camera),
                                       _I32, C.POINTER(Proposal), C.c_float, _P, _P, _I64, _P,
                                       _P, _SZ, _P]),
    "ogs_decode": (C.c_int, [_P, _P, _P, _P, _I64, C.POINTER(MLP), C.POINTER(Camera), _P, _P,
                             _I64, _P, C.POINTER(Gaussians), _P]),
    "ogs_decode_bf16": (C.c_int, [_P, _P, _P, _P, _I64, C.POINTER(MLP), C.POINTER(Camera), _P,
                                  _P, _I64, _P, C.POINTER(Gaussians), _P]),
    "ogs_project_bin": (C.c_int, [C.POINTER(Gaussians), _I64, _I32, C.POINTER(Camera), _P, _P,
                                  _P, _P, _P, _P, _P]),
    "ogs_decode_project_scratch_bytes": (_SZ, []),
    "ogs_decode_project_bf16": (C.c_int, [_P, _P, _P, _P, _I64, C.POINTER(MLP),
                                          C.POINTER(Camera), _P, _P, _I64, _P,
                                          C.POINTER(Gaussians), _P, _P, _P, _P, _P, _P, _SZ,
                                          _P]),
    "ogs_sort_bins_scratch_bytes": (_SZ, [_I32]),
    "ogs_sort_bins": (C.c_int, [_P, _P, _P, _I64, _I64, _I32, _I32, C.POINTER(TileBins), _P,
                                _P, _P, _SZ, _P]),
    "ogs_sort_scratch_bytes": (_SZ, [_I64, _I64, _I32]),
    "ogs_sort": (C.c_int, [_P, _P, _P, _P, _I64, _I64, _I32, _I32, _P, _P, _I64, _P, _P, _SZ,
                           _P]),
    "ogs_radix_sort_scratch_bytes": (_SZ, [_I64]),
    "ogs_radix_sort_pairs": (C.c_int, [_P, _P, _P, _I64, _I32, _I32, _P, _SZ, _P]),
    "ogs_blend_fwd": (C.c_int, [_P, _P, _P, _I32, _I32, C.POINTER(C.c_float * 3), _P, _P, _P,
                                _P, _P, _I32, _P, _P]),
    "ogs_blend_bwd": (C.c_int, [_P, _P, _P, _I32, _I32, C.POINTER(C.c_float * 3), _P, _P, _P,
                                _P, _P]),
    "ogs_project_bwd": (C.c_int, [C.POINTER(Gaussians), _I64, _I32, C.POINTER(Camera), _P, _P,
                                  _P, _P, _P, _P, _P]),
    "ogs_decode_bwd_scratch_bytes": (_SZ, [_I64]),
    "ogs_decode_bwd": (C.c_int, [_P, _P, _P, _P, _I64, C.POINTER(MLP), C.POINTER(Camera), _P, _P,
                                 _I64, _P, _P, _P, _P, _P, _P, _P, _P, C.POINTER(MLP), _P, _SZ,
                                 _P]),
    "ogs_decode_bwd_bf16": (C.c_int, [_P, _P, _P, _P, _I64, C.POINTER(MLP), C.POINTER(Camera), _P, _P,
                                 _I64, _P, _P, _P, _P, _P, _P, _P, _P, C.POINTER(MLP), _P, _SZ,
                                 _P]),
    "ogs_loss_l1": (C.c_int, [_P, _P, _I64, _P, _P, _P]),
    "ogs_loss_l1_ssim_scratch_bytes": (_SZ, [_I32, _I32, _I32]),
    "ogs_loss_l1_ssim": (C.c_int, [_P, _P, _I32, _I32, _I32, C.c_float, _P, _P, _P, _P, _SZ,
                                   _P]),
    "ogs_ssim_target_stats": (C.c_int, [_P, _I32, _I32, _I32, _P, _P]),
    "ogs_adam": (C.c_int, [_P, _P, _P, _P, _I64, C.c_float, C.c_float, C.c_float, C.c_float,
                           _I32, _I32, _P]),
    "ogs_scale": (C.c_int, [_P, _I64, _P, _P]),
    "ogs_scan_nonfinite": (C.c_int, [_P, _I64, _P, C.c_uint32, _P]),
    "ogs_counts_status": (C.c_int, [_P, C.c_uint32]),
    "ogs_stamp_selected": (C.c_int, [_P, _P, _I64, _P, C.c_uint32, _P]),
    "ogs_adam_rows": (C.c_int, [_P, _P, _P, _P, _I64, _I32, _P, C.c_uint32, C.c_float,
                                C.c_float, C.c_float, C.c_float, _I32, _I32, _P]),
    "ogs_radix_sort_pairs_noalloc_max_items": (_I64, []),
    "ogs_radix_sort_pairs_noalloc": (C.c_int, [_P, _P, _P, _I64, _I32, _I32, _P]),
    "ogs_proposal_gate_scratch_bytes": (_SZ, [_I64]),
    "ogs_proposal_gate": (C.c_int, [_P, _P, _P, _I64, _I32, _I32, C.POINTER(Camera),
                                    C.POINTER(Proposal), C.c_float, _P, _P, _I64, _P, _P, _P,
                                    _P, _P, _SZ, _P]),
    "ogs_proposal_gate_bf16": (C.c_int, [_P, _P, _P, _I64, _I32, _I32, C.POINTER(Camera),
                                    C.POINTER(Proposal), C.c_float, _P, _P, _I64, _P, _P, _P,
                                    _P, _P, _SZ, _P]),
    "ogs_proposal_train_scratch_bytes": (_SZ, []),
    "ogs_proposal_train": (C.c_int, [_P, _P, _P, _I64, _I32, C.POINTER(Camera),
                                     C.POINTER(Proposal), _P, _P, _P, C.c_float, C.c_float,
                                     C.POINTER(Proposal), _P, _P, _P, _SZ, _P]),
    "ogs_explicit_gaussians": (C.c_int, [_P, _P, _P, _I64, _I32, C.POINTER(Explicit),
                                         C.POINTER(Camera), _P, _P, _I64, _P,
                                         C.POINTER(Gaussians), _P]),
    "ogs_explicit_gaussians_bwd": (C.c_int, [_P, _P, _P, _I64, _I32, C.POINTER(Explicit),
                                             C.POINTER(Camera), _P, _P, _I64, _P, _P, _P, _P,
                                             _P, C.POINTER(Explicit), _P, _P, _P]),
    "ogs_count_selected": (C.c_int, [_P, _P, _P, _P]),
    "ogs_prune_scratch_bytes": (_SZ, [_I64]),
    "ogs_prune_anchors": (C.c_int, [_P, _I64, C.c_uint32, _P, _P, _P, _SZ, _P]),
    "ogs_gather_rows": (C.c_int, [_P, _P, _I64, _P, _P, _I64, _P]),
    "ogs_opacity_accumulate": (C.c_int, [_P, _P, _P, _I32, _P, _P, _P]),
    "ogs_prune_opacity_scratch_bytes": (_SZ, [_I64]),
    "ogs_prune_by_opacity": (C.c_int, [_P, _P, _I64, _I32, C.c_float, _P, _P, _P, _SZ, _P]),
    "ogs_grow_accumulate": (C.c_int, [_P, _P, _P, _P, _I32, _I32, _I32, _P, _P, _P]),
    "ogs_update_lod_bias": (C.c_int, [_P, _P, _P, _I64, _I32, _I32, _P, C.c_float, _P, _P]),
    "ogs_grow_scratch_bytes": (_SZ, [_I64, _I32]),
    "ogs_grow_anchors": (C.c_int, [_P, _P, _P, _P, _P, _P, _I64, _I32, _I32, _P, _P, _I32, _P,
                                   _P, _P, _P, _I64, _P, _P, _SZ, _P]),
    "ogs_version": (C.c_char_p, []),
}

_lib = None


def lib():
    """Load libogs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OgsError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2403_17898_gb300.build` (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(st, what):
    if st != 0:
        raise OgsError(f"{what} failed: {STATUS.get(st, st)}")


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise OgsError("expected a CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _ptr_out(t):
    """Pointer of an output that may live in pinned host memory: with unified addressing a
    pinned (page-locked) host tensor's address is valid on the device, and kernels write it
    over the host link directly."""
    if t is not None and not t.is_cuda:
        if not t.is_pinned():
            raise OgsError("expected a CUDA tensor or a pinned host tensor")
        return C.c_void_p(t.data_ptr())
    return _ptr(t)


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def camera(cam) -> Camera:
    """synth.Camera (or any object with the same fields) -> ogs_camera."""
    c = Camera()
    R = np.asarray(cam.R, np.float32).reshape(9)
    p = np.asarray(cam.campos, np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.campos[i] = float(p[i])
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    c.width, c.height = int(cam.W), int(cam.H)
    c.znear, c.d_max, c.s = (float(np.float32(v)) for v in (cam.znear, cam.d_max, cam.s))
    return c


def mlp_struct(t, k=10, F=32, H=32, app=None) -> MLP:
    """Decoder weights (dict of CUDA float32 tensors named like synth.DecoderMLP).  With
    appearance codes, ``t["w1_app"]`` is [H][A] and ``app`` the per-anchor codes [N][A] (for
    a gradient struct: their gradient arrays)."""
    m = MLP()
    for n in ("w1", "b1", "w2_op", "b2_op", "w2_col", "b2_col", "w2_cov", "b2_cov"):
        setattr(m, n, t[n].data_ptr())
    m.F, m.H, m.k = F, H, k
    if t.get("w1_app") is not None:
        assert app is not None, "appearance weights without codes"
        m.A = int(t["w1_app"].shape[1])
        m.w1_app, m.app = t["w1_app"].data_ptr(), app.data_ptr()
    return m


def gaussians_struct(t) -> Gaussians:
    g = Gaussians()
    for n in ("means", "scales", "quats", "opac", "colors"):
        setattr(g, n, t[n].data_ptr())
    return g


# ---------------------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------------------

def lod_select_scratch_bytes(N):
    return int(lib().ogs_lod_select_scratch_bytes(int(N)))


def lod_select(pos, level, dL, N, NL, k, cam, infer, sel_idx, sel_w, sel_cap, counts,
               scratch, stream=None):
    c = cam if isinstance(cam, Camera) else camera(cam)
    _check(lib().ogs_lod_select(_ptr(pos), _ptr(level), _ptr(dL), int(N), int(NL), int(k),
                                C.byref(c), int(bool(infer)), _ptr(sel_idx), _ptr(sel_w),
                                int(sel_cap), _ptr(counts), _ptr(scratch), scratch.numel(),
                                _stream(stream)), "ogs_lod_select")


def lod_select_gated_scratch_bytes(N):
    return int(lib().ogs_lod_select_gated_scratch_bytes(int(N)))


def lod_select_gated(pos, level, dL, feat, N, NL, k, cam, infer, net, p_star, sel_idx, sel_w,
                     sel_cap, counts, scratch, stream=None):
    """LOD selection and the BF16 proposal gate in one pass (ogs_lod_select_gated)."""
    c = cam if isinstance(cam, Camera) else camera(cam)
    n = net if isinstance(net, Proposal) else proposal_struct(net)
    _check(lib().ogs_lod_select_gated(_ptr(pos), _ptr(level), _ptr(dL), _ptr(feat), int(N),
                                      int(NL), int(k), C.byref(c), int(bool(infer)),
                                      C.byref(n), float(p_star), _ptr(sel_idx), _ptr(sel_w),
                                      int(sel_cap), _ptr(counts), _ptr(scratch),
                                      scratch.numel(), _stream(stream)),
           "ogs_lod_select_gated")


def decode(pos, feat, offs, lv, N, mlp, cam, sel_idx, sel_w, sel_cap, counts, out,
           stream=None):
    c = cam if isinstance(cam, Camera) else camera(cam)
    m = mlp if isinstance(mlp, MLP) else mlp_struct(mlp)
    g = out if isinstance(out, Gaussians) else gaussians_struct(out)
    _check(lib().ogs_decode(_ptr(pos), _ptr(feat), _ptr(offs), _ptr(lv), int(N), C.byref(m),
                            C.byref(c), _ptr(sel_idx), _ptr(sel_w), int(sel_cap), _ptr(counts),
                            C.byref(g), _stream(stream)), "ogs_decode")


def decode_bf16(pos, feat, offs, lv, N, mlp, cam, sel_idx, sel_w, sel_cap, counts, out,
                stream=None):
    c = cam if isinstance(cam, Camera) else camera(cam)
    m = mlp if isinstance(mlp, MLP) else mlp_struct(mlp)
    g = out if isinstance(out, Gaussians) else gaussians_struct(out)
    _check(lib().ogs_decode_bf16(_ptr(pos), _ptr(feat), _ptr(offs), _ptr(lv), int(N),
                                 C.byref(m), C.byref(c), _ptr(sel_idx), _ptr(sel_w),
                                 int(sel_cap), _ptr(counts), C.byref(g), _stream(stream)),
           "ogs_decode_bf16")


def project_bin(g, n_gauss, means_relative, cam, rec, depth_key, rect, tiles, counts=None,
                stream=None, tile_count=None):
    c = cam if isinstance(cam, Camera) else camera(cam)
    gs = g if isinstance(g, Gaussians) else gaussians_struct(g)
    _check(lib().ogs_project_bin(C.byref(gs), int(n_gauss), int(means_relative), C.byref(c),
                                 _ptr(rec), _ptr(depth_key), _ptr(rect), _ptr(tiles),
                                 _ptr(tile_count), _ptr(counts), _stream(stream)),
           "ogs_project_bin")


def decode_project_scratch_bytes():
    return int(lib().ogs_decode_project_scratch_bytes())


def tile_bins(pair_key, pair_gauss, tile_cap):
    """ogs_tile_bins of two device u32 arrays of n_tiles * tile_cap entries."""
    return TileBins(C.c_void_p(pair_key.data_ptr()), C.c_void_p(pair_gauss.data_ptr()),
                    int(tile_cap))


def decode_project_bf16(pos, feat, offs, lv, N, mlp, cam, sel_idx, sel_w, sel_cap, counts,
                        rec, depth_key, rect, tiles, scratch, out=None, tile_count=None,
                        stream=None):
    """Fused BF16 decode + projection; ``out`` (Gaussian SoA) is written only if given."""
    c = cam if isinstance(cam, Camera) else camera(cam)
    m = mlp if isinstance(mlp, MLP) else mlp_struct(mlp)
    g = None
    if out is not None:
        g = C.byref(out if isinstance(out, Gaussians) else gaussians_struct(out))
    _check(lib().ogs_decode_project_bf16(
        _ptr(pos), _ptr(feat), _ptr(offs), _ptr(lv), int(N), C.byref(m), C.byref(c),
        _ptr(sel_idx), _ptr(sel_w), int(sel_cap), _ptr(counts), g, _ptr(rec), _ptr(depth_key),
        _ptr(rect), _ptr(tiles), _ptr(tile_count), _ptr(scratch), scratch.numel(),
        _stream(stream)), "ogs_decode_project_bf16")


def sort_bins_scratch_bytes(n_tiles):
    return int(lib().ogs_sort_bins_scratch_bytes(int(n_tiles)))


def sort_bins(depth_key, rect, tiles, g_cap, n_gauss, grid_x, grid_y, bins, tile_range, counts,
              scratch, stream=None):
    """ogs_sort_bins: the tile lists in per-tile regions (``bins``, a TileBins)."""
    _check(lib().ogs_sort_bins(_ptr(depth_key), _ptr(rect), _ptr(tiles), int(g_cap),
                               int(n_gauss), int(grid_x), int(grid_y), C.byref(bins),
                               _ptr(tile_range), _ptr(counts), _ptr(scratch), scratch.numel(),
                               _stream(stream)), "ogs_sort_bins")


def sort_scratch_bytes(g_cap, pair_cap, n_tiles):
    return int(lib().ogs_sort_scratch_bytes(int(g_cap), int(pair_cap), int(n_tiles)))


def sort(depth_key, rect, tiles, g_cap, n_gauss, grid_x, grid_y, pair_gauss, tile_range,
         pair_cap, counts, scratch, stream=None, tile_count=None):
    _check(lib().ogs_sort(_ptr(depth_key), _ptr(rect), _ptr(tiles), _ptr(tile_count),
                          int(g_cap), int(n_gauss),
                          int(grid_x), int(grid_y), _ptr(pair_gauss), _ptr(tile_range),
                          int(pair_cap), _ptr(counts), _ptr(scratch), scratch.numel(),
                          _stream(stream)), "ogs_sort")


def radix_sort_scratch_bytes(n_cap):
    return int(lib().ogs_radix_sort_scratch_bytes(int(n_cap)))


def radix_sort_pairs(keys, vals, n_dev, n_cap, bit_lo, bit_hi, scratch, stream=None):
    _check(lib().ogs_radix_sort_pairs(_ptr(keys), _ptr(vals), _ptr(n_dev), int(n_cap),
                                      int(bit_lo), int(bit_hi), _ptr(scratch), scratch.numel(),
                                      _stream(stream)), "ogs_radix_sort_pairs")


def blend_fwd(rec, pair_gauss, tile_range, width, height, bg, img, T_final, n_last,
              sel_idx=None, k=10, maxc=None, n_eval=None, stream=None):
    b = (C.c_float * 3)(*[float(x) for x in bg])
    _check(lib().ogs_blend_fwd(_ptr(rec), _ptr(pair_gauss), _ptr(tile_range), int(width),
                               int(height), C.byref(b), _ptr_out(img), _ptr(T_final),
                               _ptr(n_last),
                               _ptr(n_eval), _ptr(sel_idx), int(k), _ptr(maxc),
                               _stream(stream)), "ogs_blend_fwd")


def blend_bwd(rec, pair_gauss, tile_range, width, height, bg, T_final, n_last, dimg, drec,
              stream=None):
    b = (C.c_float * 3)(*[float(x) for x in bg])
    _check(lib().ogs_blend_bwd(_ptr(rec), _ptr(pair_gauss), _ptr(tile_range), int(width),
                               int(height), C.byref(b), _ptr(T_final), _ptr(n_last), _ptr(dimg),
                               _ptr(drec), _stream(stream)), "ogs_blend_bwd")


def project_bwd(g, n_gauss, means_relative, cam, rect, drec, dmeans, dscales, dquats,
                counts=None, stream=None):
    c = cam if isinstance(cam, Camera) else camera(cam)
    gs = g if isinstance(g, Gaussians) else gaussians_struct(g)
    _check(lib().ogs_project_bwd(C.byref(gs), int(n_gauss), int(means_relative), C.byref(c),
                                 _ptr(rect), _ptr(drec), _ptr(dmeans), _ptr(dscales),
                                 _ptr(dquats), _ptr(counts), _stream(stream)), "ogs_project_bwd")


def decode_bwd_scratch_bytes(sel_cap):
    return int(lib().ogs_decode_bwd_scratch_bytes(int(sel_cap)))


def decode_bwd(pos, feat, offs, lv, N, mlp, cam, sel_idx, sel_w, sel_cap, counts, dmeans,
               dscales, dquats, drec, dfeat, doffs, dlv, dmlp, scratch, stream=None, bf16=False):
    """ogs_decode_bwd, or ogs_decode_bwd_bf16 (tensor-core products) when bf16."""
    c = cam if isinstance(cam, Camera) else camera(cam)
    m = mlp if isinstance(mlp, MLP) else mlp_struct(mlp)
    dm = dmlp if isinstance(dmlp, MLP) else mlp_struct(dmlp)
    fn = lib().ogs_decode_bwd_bf16 if bf16 else lib().ogs_decode_bwd
    _check(fn(_ptr(pos), _ptr(feat), _ptr(offs), _ptr(lv), int(N), C.byref(m),
                                C.byref(c), _ptr(sel_idx), _ptr(sel_w), int(sel_cap),
                                _ptr(counts),
                                _ptr(dmeans), _ptr(dscales), _ptr(dquats), _ptr(drec),
                                _ptr(dfeat), _ptr(doffs), _ptr(dlv), C.byref(dm), _ptr(scratch),
                                scratch.numel(), _stream(stream)),
           "ogs_decode_bwd_bf16" if bf16 else "ogs_decode_bwd")


def loss_l1(img, target, n, dimg, loss=None, stream=None):
    _check(lib().ogs_loss_l1(_ptr(img), _ptr(target), int(n), _ptr(dimg), _ptr(loss),
                             _stream(stream)), "ogs_loss_l1")


def loss_l1_ssim_scratch_bytes(C, H, W):
    return int(lib().ogs_loss_l1_ssim_scratch_bytes(int(C), int(H), int(W)))


def loss_l1_ssim(img, target, lam, dimg, loss, scratch, stream=None, target_stats=None):
    C, H, W = img.shape
    _check(lib().ogs_loss_l1_ssim(_ptr(img), _ptr(target), int(C), int(H), int(W), float(lam),
                                  _ptr(dimg), _ptr(loss), _ptr(target_stats), _ptr(scratch),
                                  scratch.numel(), _stream(stream)), "ogs_loss_l1_ssim")


def ssim_target_stats(target, stats, stream=None):
    """The target's window moments G*y, G*y^2 into stats f32[2][C][H][W]."""
    C, H, W = target.shape
    _check(lib().ogs_ssim_target_stats(_ptr(target), int(C), int(H), int(W), _ptr(stats),
                                       _stream(stream)), "ogs_ssim_target_stats")


def stamp_selected(sel_idx, counts, stamp, value, stream=None):
    _check(lib().ogs_stamp_selected(_ptr(sel_idx), _ptr(counts), sel_idx.numel(), _ptr(stamp),
                                    int(value), _stream(stream)), "ogs_stamp_selected")


def adam_rows(param, grad, m, v, stamp, value, lr, beta1, beta2, eps, step, zero_grad=True,
              stream=None):
    """Adam over the rows of param (rows = its first dimension) whose stamp equals value."""
    rows = param.shape[0]
    row_len = param[0].numel() if rows else 1
    _check(lib().ogs_adam_rows(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), int(rows),
                               int(row_len), _ptr(stamp), int(value), float(lr), float(beta1),
                               float(beta2), float(eps), int(step), int(bool(zero_grad)),
                               _stream(stream)), "ogs_adam_rows")


def scan_nonfinite(x, flag, bit=1, stream=None):
    """flag (one-element int32 device tensor) |= bit if x holds a NaN or an infinity."""
    _check(lib().ogs_scan_nonfinite(_ptr(x), x.numel(), _ptr(flag), int(bit), _stream(stream)),
           "ogs_scan_nonfinite")


def counts_status(counts_host, nonfinite=0):
    """ogs_status of a frame from its counters read back to the host (uint32 array of 8) and a
    non-finite flag word: 0 OK, 2 capacity, 3 timeout, 5 non-finite."""
    a = np.ascontiguousarray(counts_host, np.uint32)
    return int(lib().ogs_counts_status(a.ctypes.data_as(C.c_void_p), int(nonfinite)))


def scale(x, s, stream=None):
    """x *= s in place, s a one-element device tensor (no host synchronisation)."""
    _check(lib().ogs_scale(_ptr(x), x.numel(), _ptr(s), _stream(stream)), "ogs_scale")


def adam(param, grad, m, v, n, lr, beta1, beta2, eps, step, zero_grad=True, stream=None):
    _check(lib().ogs_adam(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), int(n), float(lr),
                          float(beta1), float(beta2), float(eps), int(step), int(bool(zero_grad)),
                          _stream(stream)), "ogs_adam")


def radix_sort_pairs_noalloc_max_items():
    return int(lib().ogs_radix_sort_pairs_noalloc_max_items())


def radix_sort_pairs_noalloc(keys, vals, n_dev, n_cap, bit_lo, bit_hi, stream=None):
    """Allocation-free sort: for callers that cannot give the library any scratch memory (see
    ogs_radix_sort_pairs_noalloc in include/ogs.h); calls overlapping on the GPU race."""
    _check(lib().ogs_radix_sort_pairs_noalloc(_ptr(keys), _ptr(vals), _ptr(n_dev), int(n_cap),
                                              int(bit_lo), int(bit_hi), _stream(stream)),
           "ogs_radix_sort_pairs_noalloc")


def proposal_struct(t) -> Proposal:
    """Proposal-network weights (dict of CUDA float32 tensors w1 b1 w2 b2 w3 b3)."""
    p = Proposal()
    for n in ("w1", "b1", "w2", "b2", "w3", "b3"):
        setattr(p, n, t[n].data_ptr())
    return p


def proposal_gate_scratch_bytes(sel_cap):
    return int(lib().ogs_proposal_gate_scratch_bytes(int(sel_cap)))


def proposal_gate(pos, level, feat, N, NL, k, cam, net, p_star, sel_in, w_in, sel_cap, counts,
                  sel_out, w_out, p_out, scratch, stream=None, bf16=False):
    """ogs_proposal_gate, or ogs_proposal_gate_bf16 (tensor-core scoring) when bf16."""
    c = cam if isinstance(cam, Camera) else camera(cam)
    n = net if isinstance(net, Proposal) else proposal_struct(net)
    name = "ogs_proposal_gate_bf16" if bf16 else "ogs_proposal_gate"
    _check(getattr(lib(), name)(_ptr(pos), _ptr(level), _ptr(feat), int(N), int(NL), int(k),
                                C.byref(c), C.byref(n), float(p_star), _ptr(sel_in),
                                _ptr(w_in), int(sel_cap), _ptr(counts), _ptr(sel_out),
                                _ptr(w_out), _ptr(p_out), _ptr(scratch), scratch.numel(),
                                _stream(stream)), name)


def proposal_train_scratch_bytes():
    return int(lib().ogs_proposal_train_scratch_bytes())


def proposal_train(pos, level, feat, N, NL, cam, net, sel_idx, counts, maxc, tau, grads, loss,
                   scratch, pos_weight=1.0, stream=None, dloss=None):
    c = cam if isinstance(cam, Camera) else camera(cam)
    n = net if isinstance(net, Proposal) else proposal_struct(net)
    g = grads if isinstance(grads, Proposal) else proposal_struct(grads)
    _check(lib().ogs_proposal_train(_ptr(pos), _ptr(level), _ptr(feat), int(N), int(NL),
                                    C.byref(c), C.byref(n), _ptr(sel_idx), _ptr(counts),
                                    _ptr(maxc), float(tau), float(pos_weight), C.byref(g),
                                    _ptr(loss), _ptr(dloss),
                                    _ptr(scratch), scratch.numel(), _stream(stream)),
           "ogs_proposal_train")


def version():
    return lib().ogs_version().decode()


# ---------------------------------------------------------------------------------------
# explicit Gaussians per anchor and view-frequency pruning
# ---------------------------------------------------------------------------------------

EXPLICIT_NAMES = ("log_scale", "quat", "opacity", "color_dc")


def explicit_struct(t) -> Explicit:
    """Explicit per-Gaussian attributes (dict of CUDA float32 tensors)."""
    e = Explicit()
    for n in EXPLICIT_NAMES:
        setattr(e, n, t[n].data_ptr())
    return e


def explicit_gaussians(pos, offs, lv, N, k, attr, cam, sel_idx, sel_w, sel_cap, counts, out,
                       stream=None):
    c = cam if isinstance(cam, Camera) else camera(cam)
    e = attr if isinstance(attr, Explicit) else explicit_struct(attr)
    g = out if isinstance(out, Gaussians) else gaussians_struct(out)
    _check(lib().ogs_explicit_gaussians(_ptr(pos), _ptr(offs), _ptr(lv), int(N), int(k),
                                        C.byref(e), C.byref(c), _ptr(sel_idx), _ptr(sel_w),
                                        int(sel_cap), _ptr(counts), C.byref(g), _stream(stream)),
           "ogs_explicit_gaussians")


def explicit_gaussians_bwd(pos, offs, lv, N, k, attr, cam, sel_idx, sel_w, sel_cap, counts,
                           dmeans, dscales, dquats, drec, grad, doffs, dlv, stream=None):
    c = cam if isinstance(cam, Camera) else camera(cam)
    e = attr if isinstance(attr, Explicit) else explicit_struct(attr)
    ge = grad if isinstance(grad, Explicit) else explicit_struct(grad)
    _check(lib().ogs_explicit_gaussians_bwd(_ptr(pos), _ptr(offs), _ptr(lv), int(N), int(k),
                                            C.byref(e), C.byref(c), _ptr(sel_idx), _ptr(sel_w),
                                            int(sel_cap), _ptr(counts), _ptr(dmeans),
                                            _ptr(dscales), _ptr(dquats), _ptr(drec),
                                            C.byref(ge), _ptr(doffs), _ptr(dlv), _stream(stream)),
           "ogs_explicit_gaussians_bwd")


def count_selected(sel_idx, counts, sel_count, stream=None):
    _check(lib().ogs_count_selected(_ptr(sel_idx), _ptr(counts), _ptr(sel_count),
                                    _stream(stream)), "ogs_count_selected")


def prune_scratch_bytes(N):
    return int(lib().ogs_prune_scratch_bytes(int(N)))


def prune_anchors(sel_count, N, min_count, keep_idx, n_kept, scratch, stream=None):
    _check(lib().ogs_prune_anchors(_ptr(sel_count), int(N), int(min_count), _ptr(keep_idx),
                                   _ptr(n_kept), _ptr(scratch), scratch.numel(), _stream(stream)),
           "ogs_prune_anchors")


def opacity_accumulate(opac, sel_idx, counts, k, opac_sum, opac_views, stream=None):
    _check(lib().ogs_opacity_accumulate(_ptr(opac), _ptr(sel_idx), _ptr(counts), int(k),
                                        _ptr(opac_sum), _ptr(opac_views), _stream(stream)),
           "ogs_opacity_accumulate")


def prune_opacity_scratch_bytes(N):
    return int(lib().ogs_prune_opacity_scratch_bytes(int(N)))


def prune_by_opacity(opac_sum, opac_views, N, k, tau_o, keep_idx, n_kept, scratch,
                     stream=None):
    _check(lib().ogs_prune_by_opacity(_ptr(opac_sum), _ptr(opac_views), int(N), int(k),
                                      float(tau_o), _ptr(keep_idx), _ptr(n_kept), _ptr(scratch),
                                      scratch.numel(), _stream(stream)), "ogs_prune_by_opacity")


def _host_f32(vals):
    """Host float array (kept alive by the caller) and its pointer."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(vals, dtype=np.float32))
    return a, a.ctypes.data_as(C.c_void_p)


def grow_thresholds(tau_g, beta, NL):
    """Per-level growing thresholds tau_g * 2^(beta L) and the LOD-bias thresholds 0.25 times
    those (Sec. 4.2.1), as FP32 host arrays."""
    import numpy as np
    tau = [float(tau_g) * 2.0 ** (float(beta) * L) for L in range(int(NL))]
    return np.asarray(tau, np.float32), np.asarray([0.25 * t for t in tau], np.float32)


def grow_accumulate(drec, tiles, sel_idx, counts, k, width, height, grad_acc, grad_cnt,
                    stream=None):
    _check(lib().ogs_grow_accumulate(_ptr(drec), _ptr(tiles), _ptr(sel_idx), _ptr(counts),
                                     int(k), int(width), int(height), _ptr(grad_acc),
                                     _ptr(grad_cnt), _stream(stream)), "ogs_grow_accumulate")


def update_lod_bias(level, grad_acc, grad_cnt, N, k, NL, thr_bias, eps, dL, stream=None):
    thr, tp = _host_f32(thr_bias)
    _check(lib().ogs_update_lod_bias(_ptr(level), _ptr(grad_acc), _ptr(grad_cnt), int(N),
                                     int(k), int(NL), tp, float(eps), _ptr(dL),
                                     _stream(stream)), "ogs_update_lod_bias")


def grow_scratch_bytes(N, k):
    return int(lib().ogs_grow_scratch_bytes(int(N), int(k)))


def grow_anchors(pos, level, offs, lv, grad_acc, grad_cnt, N, k, NL, tau, voxel, new_pos,
                 new_level, new_lv, parent, max_new, n_new, scratch, stream=None,
                 next_level=True):
    t, tp = _host_f32(tau)
    v, vp = _host_f32(voxel)
    _check(lib().ogs_grow_anchors(_ptr(pos), _ptr(level), _ptr(offs), _ptr(lv), _ptr(grad_acc),
                                  _ptr(grad_cnt), int(N), int(k), int(NL), tp, vp,
                                  1 if next_level else 0, _ptr(new_pos), _ptr(new_level),
                                  _ptr(new_lv), _ptr(parent), int(max_new), _ptr(n_new), _ptr(scratch), scratch.numel(),
                                  _stream(stream)), "ogs_grow_anchors")


def gather_rows(src, dst, row_bytes, idx, n_dev, n_cap, stream=None):
    _check(lib().ogs_gather_rows(_ptr(src), _ptr(dst), int(row_bytes), _ptr(idx), _ptr(n_dev),
                                 int(n_cap), _stream(stream)), "ogs_gather_rows")
