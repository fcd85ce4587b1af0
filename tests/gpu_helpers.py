"""Shared helpers of the GPU parity tests: build/load the library, move arrays, and the
knife-edge thresholds that separate decisions fixed by the inputs from those FP32 rounding
could flip (the oracle reports a margin for every discrete decision)."""
import numpy as np

# A decision whose oracle margin is below these is excluded from bit-exact comparison.
SEL_MARGIN = 1e-5        # levels (L* vs an integer) and relative frustum distance
RECT_MARGIN_PX = 2e-4    # pixels between a tile-rect edge and a value that changes it (128 px)
NEAR_MARGIN = 1e-5       # relative distance of depth to the near plane
TIE_MARGIN = 2e-6        # relative depth gap of consecutive Gaussians blended at a pixel
# relative distance of alpha to 1/255 or T to 1e-4 at a pixel.  FP32 forms the 2D conic by
# inverting the projected covariance; for elongated Gaussians (condition numbers of 1e3 and
# more, common at 1080p near the camera and at grazing angles) its relative error reaches
# ~1e-5..1e-4, which moves power = -d^T conic d / 2 by up to ~2e-4 at the 1/255 bound
# (measured: every flipped alpha decision of three 1080p city frames had a margin below
# 2.1e-4); 1e-3 keeps a factor of ~5 above that.
PX_MARGIN = 1e-3
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
    tiles that a Gaussian whose tile rectangle or near-plane test sits on a knife edge can
    gain or lose."""
    bad = fr.out["px_margin"] < PX_MARGIN
    if fr.out.get("px_tie") is not None:
        bad |= fr.out["px_tie"] < TIE_MARGIN
    tb = tiles_to_pixels(knife_tile_mask(fr, W, H, for_pixels=True), W, H)
    return bad | tb


def knife_tile_mask(fr, W, H, for_pixels=False, cam=None):
    """Tiles whose Gaussian list (or, with ``for_pixels``, whose pixels) may legitimately
    differ between FP32 and FP64:
      - a Gaussian whose tile-rectangle edge sits on a knife edge gains or loses exactly one
        tile band: tile m-1 when u - r is near 16m - 1, tile m when u + r is near 16m;
      - a Gaussian whose depth sits on the near plane can appear or vanish anywhere (it is
        huge on screen): the whole frame (such Gaussians are counted by the caller);
      - a Gaussian whose opacity sign is a knife edge (|opacity| far below 1/255, so it never
        passes the alpha test and no pixel can change) can join or leave the lists of the tiles
        its rectangle covers: those tiles (lists only; needs the view's ``cam``)."""
    gx, gy = fr.gx, fr.gy
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
    if np.any(pr["mz"] < NEAR_MARGIN):
        tile_bad[:] = True
        return tile_bad
    if not for_pixels and "op_margin" in fr.gauss:
        import oracle
        assert cam is not None, "the list mask re-projects opacity knife edges: pass cam"
        g = np.nonzero(fr.gauss["op_margin"] < 1e-5)[0]
        if len(g):
            gs = fr.gauss
            p2 = oracle.project(gs["means"][g], gs["scales"][g], gs["quats"][g],
                                np.ones(len(g)), cam)
            for x0, y0, x1, y1 in p2["rect"]:
                if x1 > x0 and y1 > y0:
                    tile_bad[max(y0 - 1, 0):min(y1 + 1, gy), max(x0 - 1, 0):min(x1 + 1, gx)] = True
    return tile_bad


def anchor_footprint_tiles(sc, mlp, cam, anchors, gx, gy):
    """Tiles that any Gaussian of the given anchors can reach: the oracle decodes them (weight
    1: a positive weight changes no opacity sign and no extent), projects them with a positive
    opacity (so that no Gaussian is culled for it) and marks their tile rectangles widened by
    one tile.  This is where a knife-edge selection decision can change lists and pixels."""
    import oracle
    out = np.zeros((gy, gx), bool)
    anchors = np.unique(np.asarray(anchors, np.int64))
    if len(anchors) == 0:
        return out
    g = oracle.decode(anchors, np.ones(len(anchors)), sc, mlp, cam)
    pr = oracle.project(g["means"], g["scales"], g["quats"], np.ones(len(g["opac"])), cam)
    for x0, y0, x1, y1 in pr["rect"]:
        if x1 > x0 and y1 > y0:
            out[max(y0 - 1, 0):min(y1 + 1, gy), max(x0 - 1, 0):min(x1 + 1, gx)] = True
    # Gaussians at or behind the near plane: their neighbourhood is unknown, take the frame
    if np.any(pr["mz"] < NEAR_MARGIN):
        out[:] = True
    return out


def tiles_to_pixels(tiles, W, H):
    return np.repeat(np.repeat(tiles, 16, 0), 16, 1)[:H, :W]


def gpu_pairs(sel_gpu, tile_range, pair_gauss, k, T):
    """GPU pairs as (tile, key) arrays in list order, keys = anchor * k + slot.  The tile
    ranges may be packed (the exclusive scan of the counts) or per-tile regions; either way
    they must lie inside pair_gauss without overlapping."""
    tr = np.asarray(tile_range).reshape(-1, 2).astype(np.int64)
    cnt = tr[:, 1] - tr[:, 0]
    ne = np.nonzero(cnt > 0)[0]
    assert np.all(cnt >= 0) and np.all(tr[ne, 1] <= len(pair_gauss))
    starts = tr[ne, 0]
    order = np.argsort(starts, kind="stable")
    assert np.all(tr[ne[order][1:], 0] >= tr[ne[order][:-1], 1])          # no overlap
    pg_all = np.asarray(pair_gauss)
    pg = (np.concatenate([pg_all[tr[t, 0]:tr[t, 1]] for t in ne]) if len(ne)
          else pg_all[:0]).astype(np.int64)
    sel_gpu = np.asarray(sel_gpu).astype(np.int64)
    return np.repeat(np.arange(T), cnt), sel_gpu[pg // k] * k + pg % k, cnt


def compare_tile_lists(fr, k, sel_gpu, tile_range, pair_gauss, knife_keys=()):
    """Per-tile Gaussian lists of the GPU against the oracle's.  Gaussians are named by
    key = anchor * k + slot, so the comparison does not depend on an anchor's rank in either
    side's selection.

    A tile is *identical* when the GPU's list equals the oracle's entry for entry.  Every
    other tile must be explained by knife edges: after removing, on both sides, the pairs of
    the Gaussians in ``knife_keys`` (those whose tile-rectangle edge, opacity sign or anchor
    selection sits on a knife edge, or whose anchors the two selections disagree on), the
    lists must be equal except for order inside groups of consecutive entries whose oracle
    depths are within TIE_MARGIN (relative) of each other (FP32 depths may tie or swap there).

    Returns (identical: bool[gy][gx], dict of counts)."""
    T = fr.gx * fr.gy
    tile_g, key_g, cnt_g = gpu_pairs(sel_gpu, tile_range, pair_gauss, k, T)
    cnt_o = np.diff(fr.start)
    tile_o = np.repeat(np.arange(T), cnt_o)
    key_o = fr.sel_idx[fr.lst // k] * k + fr.lst % k
    d_all = fr.proj["depth"][fr.lst]
    # identical tiles: equal counts and equal keys position by position
    ident = cnt_g == cnt_o
    mg, mo = ident[tile_g], ident[tile_o]
    diff = key_g[mg] != key_o[mo]
    ident[np.unique(tile_g[mg][diff])] = False
    # the other tiles, with the knife-edge Gaussians taken out on both sides
    top = max(int(key_o.max(initial=0)), int(key_g.max(initial=0))) + 1
    knife = np.zeros(top, bool)
    kk = np.asarray(sorted(knife_keys), np.int64)
    knife[kk[kk < top]] = True
    rest_o = ~ident[tile_o] & ~knife[key_o]
    rest_g = ~ident[tile_g] & ~knife[key_g]
    to, ko, do = tile_o[rest_o], key_o[rest_o], d_all[rest_o]
    tg, kg = tile_g[rest_g], key_g[rest_g]
    assert np.array_equal(np.bincount(to, minlength=T), np.bincount(tg, minlength=T)), \
        "a tile's list differs by more than its knife-edge Gaussians"
    new = np.ones(len(do), bool)
    if len(do) > 1:
        gap = np.abs(do[1:] - do[:-1]) / np.maximum(np.abs(do[:-1]), 1e-300)
        new[1:] = (to[1:] != to[:-1]) | (gap >= TIE_MARGIN)
    grp_o = np.cumsum(new) - 1
    if len(kg):
        combo_o = (to << 32) | ko
        order = np.argsort(combo_o, kind="stable")
        combo_g = (tg << 32) | kg
        pos = np.minimum(np.searchsorted(combo_o[order], combo_g), len(order) - 1)
        assert np.array_equal(combo_o[order][pos], combo_g), "a GPU pair the oracle lacks"
        grp_g = grp_o[order][pos]
        assert np.all(np.diff(grp_g) >= 0), "GPU list order differs beyond near-tied depths"
        a, b = np.lexsort((ko, grp_o)), np.lexsort((kg, grp_g))
        assert np.array_equal(ko[a], kg[b])
    stats = dict(tiles=T, identical=int(ident.sum()), pairs=int(len(key_o)),
                 knife_pairs_removed=int((~ident[tile_o] & knife[key_o]).sum()))
    return ident.reshape(fr.gy, fr.gx), stats


def knife_gaussian_keys(fr, k, W, H, differ_anchors=()):
    """Keys (anchor * k + slot) of the oracle's Gaussians whose presence in a tile list FP32
    may legitimately change: a tile-rectangle edge within rect_margin of a tile-changing value,
    an opacity sign within 1e-5 (relative) of flipping, a depth at the near plane; plus every
    slot of the anchors in ``differ_anchors`` (selection knife edges decided differently)."""
    bad = (fr.proj["mpx"] < rect_margin(W, H)) | (fr.proj["mz"] < NEAR_MARGIN)
    if "op_margin" in fr.gauss:
        bad |= fr.gauss["op_margin"] < 1e-5
    g = np.nonzero(bad)[0]
    keys = set((fr.sel_idx[g // k] * k + g % k).tolist())
    for a in np.asarray(differ_anchors, np.int64):
        keys.update(range(int(a) * k, int(a) * k + k))
    return keys


def bf16_round(a):
    """Round float32 values to bfloat16 (8 significant bits, nearest even), as float32."""
    b = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def gate_prob_bf16_model(net, X):
    """Keep probability as the tensor-core gate forms it, in FP64 otherwise: the inputs (in
    FP32), W1, the first hidden activations and W2 rounded to BF16; biases, w3 and the third
    layer exact.  What remains between this and the kernel is FP32 accumulation order and the
    kernel's exponential (~1e-6 in probability)."""
    w1, b1, w2, b2, w3, b3 = [np.asarray(a, np.float32) for a in net.arrays()]
    f = lambda a: bf16_round(a).astype(np.float64)
    a1 = f(np.asarray(X, np.float32)) @ f(w1).T + b1.astype(np.float64)
    h1 = f(np.maximum(a1, 0.0).astype(np.float32))
    a2 = h1 @ f(w2).T + b2.astype(np.float64)
    z = np.maximum(a2, 0.0) @ w3[0].astype(np.float64) + float(b3[0])
    return 1.0 / (1.0 + np.exp(-z))
