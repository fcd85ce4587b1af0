"""Shared helpers of the GPU parity tests: build/load the library, move arrays, and the
knife-edge thresholds that separate decisions fixed by the inputs from those FP32 rounding
could flip (the oracle reports a margin for every discrete decision)."""
import numpy as np

# A decision whose oracle margin is below these is excluded from bit-exact comparison.
SEL_MARGIN = 1e-5        # levels (L* vs an integer) and relative frustum distance
RECT_MARGIN_PX = 2e-4    # pixels between a tile-rect edge and a value that changes it (128 px)
NEAR_MARGIN = 1e-5       # relative distance of depth to the near plane
TIE_MARGIN = 2e-6        # relative depth gap of consecutive Gaussians blended at a pixel
PX_MARGIN = 1e-4         # relative distance of alpha to 1/255 or T to 1e-4 at a pixel
PIXEL_TOL = 1e-4         # max-abs pixel error allowed in FP32


def rect_margin(W, H):
    """FP32 error of a pixel coordinate grows with its magnitude: ~10x that error."""
    return RECT_MARGIN_PX * max(1.0, max(W, H) / 128.0)


def lib_ready():
    from paper_2403_17898_gb300 import build
    build.build()
    from paper_2403_17898_gb300 import abi
    abi.lib()
    return abi


def to_np_u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def cuda(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


def knife_pixel_mask(fr, W, H):
    """Pixels whose value may legitimately differ between FP32 and FP64: alpha/T decisions
    near their thresholds, near-tied depths among the Gaussians blended at the pixel, and
    tiles covered by a Gaussian whose tile rectangle or near-plane test sits on a knife edge
    (one tile of slack)."""
    gx, gy = fr.gx, fr.gy
    bad = fr.out["px_margin"] < PX_MARGIN
    if fr.out.get("px_tie") is not None:
        bad |= fr.out["px_tie"] < TIE_MARGIN
    tile_bad = np.zeros((gy, gx), bool)
    pr = fr.proj
    # a Gaussian whose extent edge sits on a tile-changing value can gain or lose exactly one
    # tile band: tile m-1 when u - r is near 16m - 1, tile m when u + r is near 16m
    rm = rect_margin(W, H)
    for g in np.nonzero(pr["mpx"] < rm)[0]:
        u, v = pr["uv"][g]
        r = pr["radius"][g]
        ys = (int(max((v - r) // 16, 0)), int(min((v + r) // 16 + 1, gy)))
        xs = (int(max((u - r) // 16, 0)), int(min((u + r) // 16 + 1, gx)))
        for e, off, axis in ((u - r, -1.0, 0), (u + r, 0.0, 0), (v - r, -1.0, 1), (v + r, 0.0, 1)):
            m = int(round((e - off) / 16.0))
            if abs(e - (16.0 * m + off)) >= rm:
                continue
            t = m - 1 if off < 0 else m
            if axis == 0 and 0 <= t < gx:
                tile_bad[ys[0]:ys[1], t] = True
            elif axis == 1 and 0 <= t < gy:
                tile_bad[t, xs[0]:xs[1]] = True
    # near-plane knife edges and opacity-sign knife edges: the whole neighbourhood
    g_bad = pr["mz"] < NEAR_MARGIN
    if "op_margin" in fr.gauss:
        g_bad |= fr.gauss["op_margin"] < 1e-5
    for g in np.nonzero(g_bad)[0]:
        u, v = pr["uv"][g]
        rr = pr["radius"][g] + 16
        x0, x1 = int(max((u - rr) // 16, 0)), int(min((u + rr) // 16 + 1, gx))
        y0, y1 = int(max((v - rr) // 16, 0)), int(min((v + rr) // 16 + 1, gy))
        if pr["radius"][g] <= 0:
            x0, x1, y0, y1 = 0, gx, 0, gy
        tile_bad[y0:y1, x0:x1] = True
    tb = np.repeat(np.repeat(tile_bad, 16, 0), 16, 1)[:H, :W]
    return bad | tb
