"""FP64 CPU oracle for the Octree-GS LOD renderer hot path — TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA path (``paper_2403_17898_gb300``) and
imports nothing from it.  The C library ``ogs_oracle.c`` holds the arithmetic; this module
only converts arrays to float64 / int64, calls it and composes the stages in the paper's order
(Sec. 4.1.3 selection -> Sec. 3.2 decode -> Sec. 3.1 projection, tile lists and blending).

Parity status of each function (what pins it) is stated in its docstring; every function
here is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ogs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
TILE = 16


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over pixels)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        _declare(_lib)
    return _lib


_P = C.c_void_p


def _declare(L):
    L.orc_lod_select.restype = C.c_long
    L.orc_lod_select.argtypes = [C.c_long, _P, _P, _P, C.c_int, _P, C.c_int, _P, _P, _P]
    L.orc_decode.restype = None
    L.orc_decode.argtypes = [C.c_long, _P, _P, _P, _P, C.c_int, _P, _P, C.c_int,
                             _P, _P, C.c_int, _P, _P, _P, _P, _P, _P, _P,
                             _P, _P, _P, _P, _P, _P, _P, C.c_int, _P]
    L.orc_project.restype = None
    L.orc_project.argtypes = [C.c_long] + [_P] * 12
    L.orc_tile_lists.restype = C.c_long
    L.orc_tile_lists.argtypes = [C.c_long, _P, _P, C.c_int, C.c_int, _P, _P, C.c_long, _P]
    L.orc_blend.restype = None
    L.orc_blend.argtypes = [C.c_int, C.c_int] + [_P] * 15
    L.orc_blend_bwd.restype = None
    L.orc_blend_bwd.argtypes = [C.c_int, C.c_int] + [_P] * 12
    L.orc_project_bwd.restype = None
    L.orc_project_bwd.argtypes = [C.c_long] + [_P] * 10
    L.orc_decode_bwd.restype = None
    L.orc_decode_bwd.argtypes = ([C.c_long, _P, _P, _P, _P, C.c_int, _P, _P, C.c_int,
                                  _P, _P, C.c_int, _P, _P, _P, _P, _P, _P, _P]
                                 + [_P] * 16 + [_P, C.c_int, _P, _P, _P])


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def cam_array(cam) -> np.ndarray:
    """Camera as 22 float64 (R[9], campos[3], fx, fy, cx, cy, W, H, znear, d_max, s, pad),
    upcast exactly from the float32 values both paths receive."""
    if hasattr(cam, "as_floats"):
        cam = cam.as_floats()
    return _d(np.asarray(cam, np.float32))


def grid(W, H):
    return (W + TILE - 1) // TILE, (H + TILE - 1) // TILE


# ----------------------------------------------------------------------------------------
# stages
# ----------------------------------------------------------------------------------------

def lod_select(pos, level, dL, NL, cam, infer):
    """Sec. 4.1.3 (Eq. for L_hat): selected anchor indices (ascending), weights, and the
    per-anchor decision margin.  Pinned by hand cases at d = d_max/2^m +- eps, cumulativity,
    monotonicity in distance and the s <-> distance equivalence (tests/test_oracle_select)."""
    pos, dL = _d(pos), _d(dL)
    level = np.ascontiguousarray(level, np.int32)
    N = pos.shape[0]
    idx = np.zeros(N, np.int64)
    w = np.zeros(N, np.float64)
    margin = np.zeros(N, np.float64)
    M = lib().orc_lod_select(N, _p(pos), _p(level), _p(dL), int(NL), _p(cam_array(cam)),
                             int(bool(infer)), _p(idx), _p(w), _p(margin))
    return idx[:M].copy(), w[:M].copy(), margin


def _appearance(scene, mlp):
    """Per-anchor appearance codes and the colour decoder's weights for them (Sec. 4.4), as
    (codes f64[N][A] or None, A, weights f64[H][A] or None)."""
    app = getattr(scene, "app", None)
    if app is None:
        return None, 0, None
    return _d(app), int(app.shape[1]), _d(mlp.w1_app)


def decode(sel_idx, sel_w, scene, mlp, cam):
    """Sec. 3.2 (Eq. offsets, Eq. mlp).  Gaussian g = rank*k + i.  Pinned by closed forms with
    zeroed second layers, the affine collapse when every hidden unit is active, and position
    offsets (tests/test_oracle_decode).  With appearance codes (Sec. 4.4: a learnable code per
    anchor fed to the colour MLP as an additional input), the colour decoder's first layer also
    sees the anchor's code; pinned by its equality with a decoder whose features are extended
    by the code (tests/test_oracle_appearance)."""
    sel_idx = np.ascontiguousarray(sel_idx, np.int64)
    sel_w = _d(sel_w)
    M = sel_idx.shape[0]
    k = scene.k
    F = scene.feat.shape[1]
    Hd = mlp.w1.shape[1]
    G = M * k
    out = dict(means=np.zeros((G, 3)), scales=np.zeros((G, 3)), quats=np.zeros((G, 4)),
               opac=np.zeros(G), colors=np.zeros((G, 3)), op_margin=np.zeros(G))
    ws = [_d(a) for a in mlp.arrays()]
    lib().orc_decode(M, _p(sel_idx), _p(sel_w), _p(_d(scene.pos)), _p(_d(scene.feat)), F,
                     _p(_d(scene.offs)), _p(_d(scene.lv)), k, _p(ws[0]), _p(ws[1]), Hd,
                     _p(ws[2]), _p(ws[3]), _p(ws[4]), _p(ws[5]), _p(ws[6]), _p(ws[7]),
                     _p(cam_array(cam)), _p(out["means"]), _p(out["scales"]),
                     _p(out["quats"]), _p(out["opac"]), _p(out["colors"]),
                     _p(out["op_margin"]), *_app_args(scene, mlp))
    return out


def _app_args(scene, mlp):
    app, A, w = _appearance(scene, mlp)
    return (_p(app) if app is not None else None, A, _p(w) if w is not None else None)


def project(means, scales, quats, opac, cam):
    """Sec. 3.1 (Eq. 1 and the EWA projection).  Pinned by the on-axis axis-aligned closed
    form, the 90-degree-about-z swap, radius/rect hand cases (tests/test_oracle_project)."""
    means, scales, quats, opac = _d(means), _d(scales), _d(quats), _d(opac)
    G = means.shape[0]
    o = dict(uv=np.zeros((G, 2)), conic=np.zeros((G, 3)), depth=np.zeros(G),
             radius=np.zeros(G), rect=np.zeros((G, 4), np.int32), mz=np.zeros(G),
             mpx=np.zeros(G))
    lib().orc_project(G, _p(means), _p(scales), _p(quats), _p(opac), _p(cam_array(cam)),
                      _p(o["uv"]), _p(o["conic"]), _p(o["depth"]), _p(o["radius"]),
                      _p(o["rect"]), _p(o["mz"]), _p(o["mpx"]))
    return o


def tile_lists(rect, depth, gx, gy):
    """Sec. 3.1: per tile, Gaussians whose rect covers it, ordered by (depth, id).  Pinned by
    permutation/ordering invariants and a brute-force rebuild (tests/test_oracle_lists)."""
    rect = np.ascontiguousarray(rect, np.int32)
    depth = _d(depth)
    G = rect.shape[0]
    T = gx * gy
    start = np.zeros(T + 1, np.int64)
    tie = np.zeros(T, np.float64)
    spans = np.maximum(rect[:, 2] - rect[:, 0], 0) * np.maximum(rect[:, 3] - rect[:, 1], 0)
    cap = int(spans.sum())
    lst = np.zeros(max(cap, 1), np.int64)
    P = lib().orc_tile_lists(G, _p(rect), _p(depth), int(gx), int(gy), _p(start), _p(lst),
                             cap, _p(tie))
    assert P == cap
    return start, lst[:P].copy(), tie


def blend(W, H, start, lst, uv, conic, opac, colors, bg=(0.0, 0.0, 0.0), anchor_of=None,
          n_anchors=0, depth=None):
    """Sec. 3.1 Eq. 2 with the rasterizer conventions.  Pinned by the single- and
    two-Gaussian closed forms, the clamp/skip/stop hand cases, monotone transmittance and
    input-order invariance (tests/test_oracle_blend)."""
    uv, conic, opac, colors = _d(uv), _d(conic), _d(opac), _d(colors)
    bg = _d(bg)
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    last = np.zeros((H, W), np.int32)
    m = np.zeros((H, W))
    maxc = None
    tie = None
    if depth is not None:
        depth = _d(depth)
        tie = np.zeros((H, W))
    if anchor_of is not None:
        anchor_of = np.ascontiguousarray(anchor_of, np.int64)
        maxc = np.zeros(n_anchors)
    lib().orc_blend(int(W), int(H), _p(start), _p(lst), _p(uv), _p(conic), _p(opac),
                    _p(colors), _p(bg), _p(img), _p(T), _p(last), _p(m), _p(anchor_of),
                    _p(maxc), _p(depth), _p(tie))
    return dict(img=img, T=T, last=last, px_margin=m, maxc=maxc, px_tie=tie)


def blend_bwd(W, H, start, lst, uv, conic, opac, colors, bg, dimg):
    """Analytic backward of Eq. 2 (back-to-front replay).  Pinned by central finite
    differences of ``blend`` (tests/test_oracle_grad)."""
    uv, conic, opac, colors = _d(uv), _d(conic), _d(opac), _d(colors)
    G = uv.shape[0]
    o = dict(duv=np.zeros((G, 2)), dconic=np.zeros((G, 3)), dopac=np.zeros(G),
             dcolors=np.zeros((G, 3)))
    lib().orc_blend_bwd(int(W), int(H), _p(start), _p(lst), _p(uv), _p(conic), _p(opac),
                        _p(colors), _p(_d(bg)), _p(_d(dimg)), _p(o["duv"]), _p(o["dconic"]),
                        _p(o["dopac"]), _p(o["dcolors"]))
    return o


def project_bwd(means, scales, quats, rect, cam, duv, dconic):
    """Analytic backward of the EWA projection.  Pinned by finite differences."""
    means, scales, quats = _d(means), _d(scales), _d(quats)
    G = means.shape[0]
    o = dict(dmeans=np.zeros((G, 3)), dscales=np.zeros((G, 3)), dquats=np.zeros((G, 4)))
    lib().orc_project_bwd(G, _p(means), _p(scales), _p(quats),
                          _p(np.ascontiguousarray(rect, np.int32)), _p(cam_array(cam)),
                          _p(_d(duv)), _p(_d(dconic)), _p(o["dmeans"]), _p(o["dscales"]),
                          _p(o["dquats"]))
    return o


def decode_bwd(sel_idx, sel_w, scene, mlp, cam, g):
    """Analytic backward of the decoders.  Pinned by finite differences."""
    sel_idx = np.ascontiguousarray(sel_idx, np.int64)
    sel_w = _d(sel_w)
    M = sel_idx.shape[0]
    k = scene.k
    N, F = scene.feat.shape
    Hd = mlp.w1.shape[1]
    ws = [_d(a) for a in mlp.arrays()]
    o = dict(dfeat=np.zeros((N, F)), doffs=np.zeros((N, k, 3)), dlv=np.zeros((N, 3)))
    names = ["dw1", "db1", "dw2_op", "db2_op", "dw2_col", "db2_col", "dw2_cov", "db2_cov"]
    for n, a in zip(names, mlp.arrays()):
        o[n] = np.zeros(a.shape)
    app, A, w1app = _appearance(scene, mlp)
    if A:
        o["dapp"] = np.zeros((N, A))
        o["dw1_app"] = np.zeros(w1app.shape)
    lib().orc_decode_bwd(M, _p(sel_idx), _p(sel_w), _p(_d(scene.pos)), _p(_d(scene.feat)), F,
                         _p(_d(scene.offs)), _p(_d(scene.lv)), k, _p(ws[0]), _p(ws[1]), Hd,
                         _p(ws[2]), _p(ws[3]), _p(ws[4]), _p(ws[5]), _p(ws[6]), _p(ws[7]),
                         _p(cam_array(cam)), _p(_d(g["dmeans"])), _p(_d(g["dscales"])),
                         _p(_d(g["dquats"])), _p(_d(g["dopac"])), _p(_d(g["dcolors"])),
                         _p(o["dfeat"]), _p(o["doffs"]), _p(o["dlv"]),
                         *[_p(o[n]) for n in names],
                         _p(app) if A else None, A, _p(w1app) if A else None,
                         _p(o["dapp"]) if A else None, _p(o["dw1_app"]) if A else None)
    return o


def stable_sort_pairs(keys, vals):
    """Stable sort of (key, value) pairs by key: a library sort is the whole definition.
    Pinned by ordering/permutation/stability properties (tests/test_oracle_lists)."""
    order = np.argsort(np.asarray(keys), kind="stable")
    return np.asarray(keys)[order], np.asarray(vals)[order]


# ----------------------------------------------------------------------------------------
# composed forward / backward
# ----------------------------------------------------------------------------------------

@dataclass
class Frame:
    sel_idx: np.ndarray
    sel_w: np.ndarray
    sel_margin: np.ndarray
    gauss: dict
    proj: dict
    start: np.ndarray
    lst: np.ndarray
    tie: np.ndarray
    out: dict
    gx: int
    gy: int


def render(scene, mlp, cam, infer=True, bg=(0.0, 0.0, 0.0), want_maxc=False, gate=None):
    """The whole forward pass of one view, stage by stage.  ``gate = (net, p_star)`` applies
    the learned anchor-visibility proposal after the LOD rule: of the selected anchors only
    those whose keep probability is at least p_star go on to decoding (order kept)."""
    sel_idx, sel_w, margin = lod_select(scene.pos, scene.level, scene.dL, scene.NL, cam, infer)
    if gate is not None:
        net, p_star = gate
        p, _ = proposal_forward(net, proposal_inputs(scene.pos, scene.level, scene.feat,
                                                     scene.NL, sel_idx, cam))
        keep = p >= p_star
        sel_idx, sel_w = sel_idx[keep], sel_w[keep]
    g = decode(sel_idx, sel_w, scene, mlp, cam)
    pr = project(g["means"], g["scales"], g["quats"], g["opac"], cam)
    gx, gy = grid(cam.W, cam.H)
    start, lst, tie = tile_lists(pr["rect"], pr["depth"], gx, gy)
    anchor_of = np.repeat(sel_idx, scene.k) if want_maxc else None
    out = blend(cam.W, cam.H, start, lst, pr["uv"], pr["conic"], g["opac"], g["colors"], bg,
                anchor_of=anchor_of, n_anchors=scene.N, depth=pr["depth"])
    return Frame(sel_idx, sel_w, margin, g, pr, start, lst, tie, out, gx, gy)


def render_grad(scene, mlp, cam, fr: Frame, dimg, bg=(0.0, 0.0, 0.0)):
    """Backward of ``render`` for a given dL/dimage: blend -> projection -> decoders."""
    g, pr = fr.gauss, fr.proj
    gb = blend_bwd(cam.W, cam.H, fr.start, fr.lst, pr["uv"], pr["conic"], g["opac"],
                   g["colors"], bg, dimg)
    pb = project_bwd(g["means"], g["scales"], g["quats"], pr["rect"], cam, gb["duv"],
                     gb["dconic"])
    per_g = dict(dmeans=pb["dmeans"], dscales=pb["dscales"], dquats=pb["dquats"],
                 dopac=gb["dopac"], dcolors=gb["dcolors"])
    db = decode_bwd(fr.sel_idx, fr.sel_w, scene, mlp, cam, per_g)
    db.update(per_gauss=per_g, blend=gb)
    return db


def l1_loss(img, target):
    """Mean absolute error over all channels and pixels, and its gradient."""
    diff = _d(img) - _d(target)
    return float(np.abs(diff).mean()), np.sign(diff) / diff.size


def adam(param, grad, m, v, lr, beta1, beta2, eps, step):
    """One Adam update (the optimiser of the training loop; FP64): returns new (param, m, v).
    Pinned by its first-step closed form p - lr * g / (|g| + eps') (tests/test_oracle_train)."""
    param, grad, m, v = _d(param), _d(grad), _d(m), _d(v)
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v


def adam_rows(param, grad, m, v, rows, lr, beta1, beta2, eps, step):
    """Adam over touched rows only (the optimiser step over the anchors a training step's
    views selected): the rows listed in ``rows`` get one ``adam`` update with the bias
    correction of the global step count; every other row keeps its parameters and moments
    (lazy Adam).  Returns new (param, m, v).  Pinned by: all rows = dense Adam, no rows = no
    change, and a row skipped on one step against the recursion written out by hand
    (tests/test_oracle_train)."""
    P, M, V = _d(param).copy(), _d(m).copy(), _d(v).copy()
    r = np.asarray(rows, np.int64)
    if len(r):
        P[r], M[r], V[r] = adam(P[r], _d(grad)[r], M[r], V[r], lr, beta1, beta2, eps, step)
    return P, M, V


# ----------------------------------------------------------------------------------------
# anchor-visibility proposal network (learned gate in front of decoding)
# ----------------------------------------------------------------------------------------

def proposal_inputs(pos, level, feat, NL, sel_idx, cam):
    """Per selected anchor: [f_v, L/(NL-1), unit viewing direction in the camera frame
    R (x - c)/|x - c|, ln(d/d_max)]."""
    c = cam_array(cam)
    R, campos, d_max = c[0:9].reshape(3, 3), c[9:12], c[19]
    p = _d(pos)[sel_idx] - campos
    d = np.linalg.norm(p, axis=1, keepdims=True)
    lev = np.asarray(level, np.float64)[sel_idx][:, None] / max(NL - 1, 1)
    return np.concatenate([_d(feat)[sel_idx], lev, (p @ R.T) / d, np.log(d / d_max)], 1)


def proposal_forward(net, X):
    """3-layer MLP (ReLU, ReLU, sigmoid): keep probability per row of X, plus the hidden
    pre-activations.  Pinned by closed forms and finite differences (tests/test_oracle_proposal)."""
    w1, b1, w2, b2, w3, b3 = [_d(a) for a in net.arrays()]
    a1 = X @ w1.T + b1
    h1 = np.maximum(a1, 0)
    a2 = h1 @ w2.T + b2
    h2 = np.maximum(a2, 0)
    z = (h2 @ w3.T + b3)[:, 0]
    p = 1.0 / (1.0 + np.exp(-z))
    return p, dict(a1=a1, h1=h1, a2=a2, h2=h2, z=z)


def proposal_bce_grad(net, X, y, pos_weight=1.0):
    """Mean weighted binary cross-entropy of the keep probability against labels y in {0, 1}
    (positives weighted by pos_weight), and its gradients w.r.t. every weight (analytic
    backward; dL/dz = w_y (p - y) / n)."""
    w1, b1, w2, b2, w3, b3 = [_d(a) for a in net.arrays()]
    p, t = proposal_forward(net, X)
    y = np.asarray(y, np.float64)
    n = len(y)
    eps = 1e-300
    wy = np.where(y > 0, pos_weight, 1.0)
    loss = float(-np.mean(wy * (y * np.log(np.maximum(p, eps)) +
                                (1 - y) * np.log(np.maximum(1 - p, eps)))))
    dz = wy * (p - y) / n
    dw3 = dz[None, :] @ t["h2"]
    db3 = np.array([dz.sum()])
    dh2 = dz[:, None] * w3[0][None, :] * (t["a2"] > 0)
    dw2 = dh2.T @ t["h1"]
    db2 = dh2.sum(0)
    dh1 = (dh2 @ w2) * (t["a1"] > 0)
    dw1 = dh1.T @ X
    db1 = dh1.sum(0)
    return loss, dict(w1=dw1, b1=db1, w2=dw2, b2=db2, w3=dw3, b3=db3)


# ----------------------------------------------------------------------------------------
# SSIM term of the photometric loss (Sec. 5.1.5: 0.8 L1 + 0.2 D-SSIM)
# ----------------------------------------------------------------------------------------

SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2


def gaussian_window(size=11, sigma=1.5):
    """Normalised 1D Gaussian window; the 2D window is its outer product."""
    x = np.arange(size) - size // 2
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    return g / g.sum()


def _blur(img, win):
    """Separable 2D correlation with zero padding ('same' size), per channel."""
    r = len(win) // 2
    out = np.zeros_like(img)
    tmp = np.zeros_like(img)
    H, W = img.shape[-2:]
    for i, w in enumerate(win):
        o = i - r
        # horizontal: tmp[:, y, x] += w * img[:, y, x + o]
        xs = slice(max(0, -o), min(W, W - o))
        xd = slice(max(0, o), min(W, W + o))
        tmp[..., :, xs] += w * img[..., :, xd]
    for i, w in enumerate(win):
        o = i - r
        ys = slice(max(0, -o), min(H, H - o))
        yd = slice(max(0, o), min(H, H + o))
        out[..., ys, :] += w * tmp[..., yd, :]
    return out


def ssim(x, y, win=None):
    """Mean SSIM over channels and pixels (Wang et al. 2004 form, Gaussian window, zero padded)
    and dSSIM/dx.  Pinned by SSIM(x, x) = 1, the constant-image closed form and finite
    differences (tests/test_oracle_ssim)."""
    win = gaussian_window() if win is None else win
    x, y = _d(x), _d(y)
    mx, my = _blur(x, win), _blur(y, win)
    exx, eyy, exy = _blur(x * x, win), _blur(y * y, win), _blur(x * y, win)
    sx, sy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    A1, A2 = 2 * mx * my + SSIM_C1, 2 * sxy + SSIM_C2
    B1, B2 = mx * mx + my * my + SSIM_C1, sx + sy + SSIM_C2
    S = A1 * A2 / (B1 * B2)
    n = S.size
    dS = 1.0 / n                       # d mean(S) / d S_p
    g1 = dS * S * (2 * my / A1 - 2 * my / A2 - 2 * mx / B1 + 2 * mx / B2)
    g2 = dS * S * (-1.0 / B2)
    g3 = dS * S * (2.0 / A2)
    grad = _blur(g1, win) + 2 * x * _blur(g2, win) + y * _blur(g3, win)
    return float(S.mean()), grad


def photometric_loss(img, target, lam=0.2):
    """(1 - lam) L1 + lam (1 - SSIM) and its gradient w.r.t. img."""
    l1, g1 = l1_loss(img, target)
    s, gs = ssim(img, target)
    return (1 - lam) * l1 + lam * (1 - s), (1 - lam) * g1 - lam * gs


# ----------------------------------------------------------------------------------------
# view-frequency pruning (Sec. 4.2.2 "Anchor Pruning")
# ----------------------------------------------------------------------------------------

def view_frequency_counts(N, selections):
    """Number of training views in which each of the N anchors was selected: the numerator
    of the view frequency (the probability that an anchor is selected in the training
    views).  ``selections`` holds one array of selected anchor indices per view.  Pinned by
    hand-built selections and by recounting oracle selections anchor by anchor."""
    count = np.zeros(N, np.int64)
    for sel in selections:
        for j in np.asarray(sel, np.int64):
            count[j] += 1
    return count


def prune_by_view_frequency(count, n_views, tau_v):
    """Anchors kept by view-frequency pruning: those whose frequency count / n_views is not
    below the visibility threshold tau_v, in ascending index order.  Pinned by hand cases at
    the threshold (a frequency equal to tau_v is kept), tau_v = 0 (all kept) and tau_v > 1
    (none kept), and monotonicity in tau_v."""
    count = np.asarray(count, np.int64)
    freq = count.astype(np.float64) / float(n_views)
    return np.nonzero(~(freq < float(tau_v)))[0].astype(np.int64)


def min_count_for(n_views, tau_v):
    """Smallest selection count whose frequency count / n_views is not below tau_v (the
    integer form of the pruning test, evaluated with the same float64 division)."""
    c = int(np.ceil(float(tau_v) * n_views))
    while c > 0 and not ((c - 1) / float(n_views) < float(tau_v)):
        c -= 1
    while c / float(n_views) < float(tau_v):
        c += 1
    return c


def opacity_accumulate(N, k, sel_idx, opac, acc=None, views=None):
    """One training view's contribution to the average-opacity statistic of anchor pruning
    (Sec. 4.2.2): every selected anchor adds the opacities of its k generated Gaussians, a
    dropped Gaussian (opacity <= 0) counting as 0, and one view.  Pinned by hand values."""
    acc = np.zeros(N) if acc is None else acc
    views = np.zeros(N, np.int64) if views is None else views
    opac = np.asarray(opac, np.float64).reshape(-1, k)
    for r, j in enumerate(np.asarray(sel_idx, np.int64)):
        acc[j] += np.maximum(opac[r], 0.0).sum()
        views[j] += 1
    return acc, views


def prune_by_opacity(acc, views, k, tau_o):
    """Anchors kept by opacity pruning (Sec. 4.2.2): an anchor seen in at least one counted
    view is removed when the average opacity of the Gaussians it generated, acc / (views k)
    (FP32 sum and quotient), is below tau_o; anchors no view selected are kept (view frequency
    handles them).  Ascending index order.  Pinned by hand cases at the threshold."""
    acc = np.asarray(acc, np.float32)
    views = np.asarray(views, np.int64)
    keep = []
    for j in range(len(acc)):
        if views[j] > 0 and np.float32(acc[j]) / np.float32(views[j] * k) < np.float32(tau_o):
            continue
        keep.append(j)
    return np.asarray(keep, np.int64)


# ----------------------------------------------------------------------------------------
# anchor growing and the LOD-bias update (Sec. 4.2.1)
# ----------------------------------------------------------------------------------------
#
# Decisions that floating point takes (threshold tests, the voxel a position falls in) are
# taken in FP32, the precision of the CUDA path, with one IEEE operation per step (product,
# sum, quotient, each correctly rounded), so that both sides decide identically.  The
# accumulated gradient norms themselves are FP64.

VOX_BITS = 20                       # bits per voxel coordinate in a key
VOX_LIM = 1 << (VOX_BITS - 1)       # coordinates lie in [-VOX_LIM, VOX_LIM)


def grow_thresholds(tau_g, beta, NL):
    """Per-level growing thresholds tau_g * 2^(beta L) (Sec. 4.2.1) and the LOD-bias
    thresholds 0.25 tau_g * 2^(beta L), both rounded to FP32.  Pinned by tau[0] = tau_g,
    the ratio 2^beta between levels and the factor 0.25."""
    L = np.arange(NL, dtype=np.float64)
    tau = float(tau_g) * np.power(2.0, float(beta) * L)
    return tau.astype(np.float32), (0.25 * tau).astype(np.float32)


def grow_accumulate(N, k, sel_idx, drec, tiles, W, H, acc=None, cnt=None):
    """One view's contribution to the growing statistics: for every Gaussian g (g = r k + i
    of the r-th selected anchor) whose projection touches a tile, the norm of its view-space
    mean gradient (dL/du, dL/dv scaled by W/2 and H/2 to normalised device coordinates, the
    units of the cited 3D-GS thresholds) is added to acc[anchor][i] and cnt[anchor][i] += 1.
    Pinned by hand values (a 3-4-5 gradient) and invisible Gaussians adding nothing."""
    acc = np.zeros((N, k)) if acc is None else acc
    cnt = np.zeros((N, k), np.int64) if cnt is None else cnt
    drec = np.asarray(drec, np.float64)
    tiles = np.asarray(tiles)
    G = len(sel_idx) * k
    for g in range(G):
        if tiles[g] <= 0:
            continue
        j, i = int(sel_idx[g // k]), g % k
        acc[j, i] += np.hypot(drec[g, 0] * (W / 2.0), drec[g, 1] * (H / 2.0))
        cnt[j, i] += 1
    return acc, cnt


def _avg_f32(acc, cnt):
    """FP32 average of FP32 sums: acc / cnt, one correctly rounded division."""
    return np.float32(acc) / np.float32(cnt)


def lod_bias_update(level, acc, cnt, thr_bias, eps, dL):
    """LOD-bias update (Sec. 4.2.1): an anchor's gradient grad_v is the average over all its
    Gaussians' counted views (sum of its k accumulated norms, summed in slot order in FP32,
    over the sum of their counts); anchors of level L with grad_v > thr_bias[L] get
    dL += eps (FP32).  Pinned by hand cases on both sides of the threshold and anchors that
    no view saw."""
    acc = np.asarray(acc, np.float32)
    cnt = np.asarray(cnt, np.int64)
    out = np.array(dL, np.float32, copy=True)
    for j in range(acc.shape[0]):
        s = np.float32(0.0)
        for i in range(acc.shape[1]):
            s = np.float32(s + acc[j, i])
        c = int(cnt[j].sum())
        if c > 0 and _avg_f32(s, c) > np.float32(thr_bias[int(level[j])]):
            out[j] = np.float32(out[j] + np.float32(eps))
    return out


def voxel_of(p, vs):
    """Voxel index of a point on a grid of spacing vs: the nearest grid point rint(p / vs)
    per axis (Eq. for V_L: voxels are centred on the grid points; ties to even), the quotient
    rounded to FP32 first; None if a coordinate falls outside [-VOX_LIM, VOX_LIM)."""
    v = np.rint(np.asarray(p, np.float32) / np.float32(vs)).astype(np.int64)
    if np.any(v < -VOX_LIM) or np.any(v >= VOX_LIM):
        return None
    return tuple(int(x) for x in v)


def progressive_schedule(NL, total, omega):
    """Progressive training (Sec. 4.3): training starts with levels 0 .. floor(NL / 2) active
    and activates one more level at a time; level i is the finest active level for N_i
    iterations with N_{i-1} = omega N_i and the N_i summing to `total`.  Returns the list of
    (first iteration, finest active level) stages, the last level staying active after
    `total`.  Pinned by the sum, the ratios and the start level."""
    s0 = NL // 2
    levels = list(range(s0, NL))
    n_last = float(total) / sum(float(omega) ** m for m in range(len(levels)))
    lengths = [n_last * float(omega) ** (NL - 1 - i) for i in levels]
    stages, start = [], 0.0
    for i, n in zip(levels, lengths):
        stages.append((int(round(start)), i))
        start += n
    return stages


def active_level(stages, it):
    """Finest active level at iteration `it` of a progressive schedule."""
    lvl = stages[0][1]
    for first, L in stages:
        if it >= first:
            lvl = L
    return lvl


def grow_anchors(pos, level, offs, lv, acc, cnt, NL, tau, voxel, next_level=True):
    """Anchor growing (Sec. 4.2.1, next-level growth).  Every Gaussian (j, i) seen in at least
    one view, with FP32 average gradient g = acc / cnt and anchor level L, proposes a voxel:
    at level L + 1 if L + 1 < NL and g > tau[L + 1], else at level L if g > tau[L], holding
    its position mu = pos_j + offs_ji * lv_j (FP32 product, then sum).  A proposal becomes an
    anchor if no anchor of that level occupies that voxel and no proposal with a smaller index
    j k + i took it first.  Returns (new_pos at the voxel centres = grid points, new_level,
    new_lv = voxel size per axis, parent = proposing anchor), in increasing proposal index.  Pinned by hand
    cases (each branch of the level rule, the finest level, occupied voxels, duplicate
    proposals, unseen Gaussians, the centre formula) and a brute-force loop on small scenes.
    next_level=False grows at the Gaussian's own level only (the progressive stage of
    Sec. 4.3 disables the next-level operator)."""
    pos = np.asarray(pos, np.float32)
    offs = np.asarray(offs, np.float32)
    lv = np.asarray(lv, np.float32)
    acc = np.asarray(acc, np.float32)
    cnt = np.asarray(cnt, np.int64)
    N, k = acc.shape
    occupied = set()
    for j in range(N):
        L = int(level[j])
        v = voxel_of(pos[j], voxel[L])
        if v is not None:
            occupied.add((L,) + v)
    taken = set()
    new_pos, new_level, new_lv, parent = [], [], [], []
    for j in range(N):
        L = int(level[j])
        for i in range(k):
            if cnt[j, i] <= 0:
                continue
            g = _avg_f32(acc[j, i], cnt[j, i])
            if next_level and L + 1 < NL and g > np.float32(tau[L + 1]):
                T = L + 1
            elif g > np.float32(tau[L]):
                T = L
            else:
                continue
            mu = (pos[j] + offs[j, i] * lv[j]).astype(np.float32)
            v = voxel_of(mu, voxel[T])
            if v is None:
                continue
            key = (T,) + v
            if key in occupied or key in taken:
                continue
            taken.add(key)
            vs = np.float32(voxel[T])
            new_pos.append(np.asarray(v, np.float32) * vs)
            new_level.append(T)
            new_lv.append([vs, vs, vs])
            parent.append(j)
    return (np.asarray(new_pos, np.float32).reshape(-1, 3), np.asarray(new_level, np.uint8),
            np.asarray(new_lv, np.float32).reshape(-1, 3), np.asarray(parent, np.int64))


def _pack_keys(T, v):
    """Voxel keys (level, x, y, z) as unsigned 64-bit integers (one per row)."""
    u = (np.asarray(v, np.int64) + VOX_LIM).astype(np.uint64)
    return ((np.asarray(T, np.uint64) << np.uint64(60)) | (u[..., 0] << np.uint64(40)) |
            (u[..., 1] << np.uint64(20)) | u[..., 2])


def grow_anchors_vectorized(pos, level, offs, lv, acc, cnt, NL, tau, voxel, next_level=True):
    """grow_anchors with array operations (the same FP32 steps; set membership by np.isin,
    first proposal per voxel by np.unique over proposals in index order), for scenes of
    millions of anchors.  Pinned against the loop form grow_anchors on seeded scenes."""
    pos = np.asarray(pos, np.float32)
    offs = np.asarray(offs, np.float32)
    lv = np.asarray(lv, np.float32)
    acc = np.asarray(acc, np.float32)
    cnt = np.asarray(cnt, np.int64)
    lev = np.asarray(level, np.int64)
    N, k = acc.shape
    vox = np.asarray(voxel, np.float32)
    t32 = np.asarray(tau, np.float32)

    def in_range(v):
        return np.all((v >= -VOX_LIM) & (v < VOX_LIM), axis=-1)

    ev = np.rint(pos / vox[lev][:, None]).astype(np.int64)
    eok = in_range(ev)
    ekeys = _pack_keys(lev[eok], ev[eok])
    seen = cnt > 0
    g = np.zeros((N, k), np.float32)
    np.divide(acc, cnt.astype(np.float32), out=g, where=seen)
    Lj = np.broadcast_to(lev[:, None], (N, k))
    up = (Lj + 1 < NL) & (g > t32[np.minimum(Lj + 1, NL - 1)]) & bool(next_level)
    same = ~up & (g > t32[Lj])
    T = np.where(up, Lj + 1, Lj)
    prop = seen & (up | same)
    mu = pos[:, None, :] + offs * lv[:, None, :]
    pv = np.rint(mu / vox[T][..., None]).astype(np.int64)
    prop &= in_range(pv)
    cid = np.nonzero(prop.ravel())[0]
    keys = _pack_keys(T.ravel()[cid], pv.reshape(-1, 3)[cid])
    fresh = ~np.isin(keys, ekeys)
    cid, keys = cid[fresh], keys[fresh]
    _, first = np.unique(keys, return_index=True)
    win = cid[np.sort(first)]
    Tw = T.ravel()[win]
    vs = vox[Tw]
    new_pos = pv.reshape(-1, 3)[win].astype(np.float32) * vs[:, None]
    return (new_pos.astype(np.float32), Tw.astype(np.uint8),
            np.repeat(vs[:, None], 3, axis=1).astype(np.float32), (win // k).astype(np.int64))


# ----------------------------------------------------------------------------------------
# explicit Gaussians per anchor ("Our-3D-GS", Sec. 5 and Sec. 3.2 Eq. offsets)
# ----------------------------------------------------------------------------------------

SH_C0 = 0.28209479177387814          # degree-0 spherical harmonic, 1 / (2 sqrt(pi))


def explicit_gaussians(sel_idx, sel_w, scene, attr):
    """The k explicit 3D Gaussians of every selected anchor, in place of the decoders:
    position x_v + O_i * l_v (Eq. offsets), scale exp(s_i), unit quaternion q_i / |q_i|
    (w, x, y, z), opacity sigmoid(a_i) times the anchor's LOD weight, colour from the
    degree-0 spherical harmonic max(0, SH_C0 f_i + 1/2) (the cited 3D-GS activations).
    ``attr`` holds log_scale [N][k][3], quat [N][k][4], opacity [N][k] (logits) and
    color_dc [N][k][3].  World-space means.  Pinned by activation closed forms and the
    offset composition."""
    sel = np.asarray(sel_idx, np.int64)
    w = _d(sel_w)
    k = scene.k
    pos, offs, lv = _d(scene.pos)[sel], _d(scene.offs)[sel], _d(scene.lv)[sel]
    means = pos[:, None, :] + offs * lv[:, None, :]
    scales = np.exp(_d(attr["log_scale"])[sel])
    q = _d(attr["quat"])[sel]
    quats = q / np.linalg.norm(q, axis=-1, keepdims=True)
    opac = w[:, None] / (1.0 + np.exp(-_d(attr["opacity"])[sel]))
    colors = np.maximum(SH_C0 * _d(attr["color_dc"])[sel] + 0.5, 0.0)
    M = len(sel)
    return dict(means=means.reshape(M * k, 3), scales=scales.reshape(M * k, 3),
                quats=quats.reshape(M * k, 4), opac=opac.reshape(M * k),
                colors=colors.reshape(M * k, 3))


def explicit_gaussians_bwd(sel_idx, sel_w, scene, attr, g):
    """Gradients of explicit_gaussians for per-Gaussian upstream gradients g (dmeans,
    dscales, dquats, dopac, dcolors): d log_scale, d quat, d opacity logit, d color_dc and
    the offsets / scalings terms (doffs, dlv), accumulated per anchor.  Pinned by central
    finite differences of explicit_gaussians."""
    sel = np.asarray(sel_idx, np.int64)
    w = _d(sel_w)
    k = scene.k
    N = scene.N
    M = len(sel)
    sh = lambda a, c: _d(a).reshape(M, k, c)
    offs, lv = _d(scene.offs)[sel], _d(scene.lv)[sel]
    s = _d(attr["log_scale"])[sel]
    q = _d(attr["quat"])[sel]
    a = _d(attr["opacity"])[sel]
    f = _d(attr["color_dc"])[sel]
    dmeans, dscales, dquats = sh(g["dmeans"], 3), sh(g["dscales"], 3), sh(g["dquats"], 4)
    dopac, dcolors = _d(g["dopac"]).reshape(M, k), sh(g["dcolors"], 3)
    out = dict(dlog_scale=np.zeros((N, k, 3)), dquat=np.zeros((N, k, 4)),
               dopacity=np.zeros((N, k)), dcolor_dc=np.zeros((N, k, 3)),
               doffs=np.zeros((N, k, 3)), dlv=np.zeros((N, 3)))
    n = np.linalg.norm(q, axis=-1, keepdims=True)
    qn = q / n
    sg = 1.0 / (1.0 + np.exp(-a))
    np.add.at(out["dlog_scale"], sel, dscales * np.exp(s))
    np.add.at(out["dquat"], sel, (dquats - qn * (qn * dquats).sum(-1, keepdims=True)) / n)
    np.add.at(out["dopacity"], sel, dopac * w[:, None] * sg * (1.0 - sg))
    np.add.at(out["dcolor_dc"], sel, np.where(SH_C0 * f + 0.5 > 0.0, dcolors * SH_C0, 0.0))
    np.add.at(out["doffs"], sel, dmeans * lv[:, None, :])
    np.add.at(out["dlv"], sel, (dmeans * offs).sum(1))
    return out


def render_explicit(scene, attr, cam, infer=True, bg=(0.0, 0.0, 0.0)):
    """The forward pass of one view with explicit Gaussians in place of the decoders."""
    sel_idx, sel_w, margin = lod_select(scene.pos, scene.level, scene.dL, scene.NL, cam, infer)
    g = explicit_gaussians(sel_idx, sel_w, scene, attr)
    pr = project(g["means"], g["scales"], g["quats"], g["opac"], cam)
    gx, gy = grid(cam.W, cam.H)
    start, lst, tie = tile_lists(pr["rect"], pr["depth"], gx, gy)
    out = blend(cam.W, cam.H, start, lst, pr["uv"], pr["conic"], g["opac"], g["colors"], bg,
                depth=pr["depth"])
    return Frame(sel_idx, sel_w, margin, g, pr, start, lst, tie, out, gx, gy)
