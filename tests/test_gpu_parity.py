"""GPU parity: every C-ABI stage against the FP64 oracle on the same seeded inputs.

Integer work (selection, tile rectangles, sorted lists, tile ranges, n_last) must match
bit-exactly wherever the oracle's margin shows the decision is fixed by the inputs;
floating-point outputs must agree within FP32 tolerances (pixels 1e-4 max-abs).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import (NEAR_MARGIN, PIXEL_TOL, PX_MARGIN, SEL_MARGIN, cuda, knife_pixel_mask,
                         lib_ready, rect_margin, to_np_u32)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    return lib_ready()


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _counts(abi, t):
    v = to_np_u32(t)
    return dict(zip(abi.COUNT_FIELDS, v.tolist()))


# ---------------------------------------------------------------------------------------
# lod_select
# ---------------------------------------------------------------------------------------

def _gpu_select(abi, torch, sc, cam, infer, cap=None):
    N = sc.N
    cap = N if cap is None else cap
    sel = torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda")
    w = torch.zeros(max(cap, 1), device="cuda")
    counts = torch.zeros(8, dtype=torch.int32, device="cuda")
    scr = torch.empty(abi.lod_select_scratch_bytes(N), dtype=torch.uint8, device="cuda")
    abi.lod_select(cuda(sc.pos), cuda(sc.level), cuda(sc.dL), N, sc.NL, sc.k, cam, infer,
                   sel, w, cap, counts, scr)
    torch.cuda.synchronize()
    c = _counts(abi, counts)
    assert c["timeout"] == 0                 # no look-back wait expired
    M = c["n_selected"]
    return to_np_u32(sel)[:M].astype(np.int64), w.cpu().numpy()[:M], c


def _check_select(abi, torch, sc, cam, infer):
    idx_o, w_o, margin = oracle.lod_select(sc.pos, sc.level, sc.dL, sc.NL, cam, infer)
    idx_g, w_g, c = _gpu_select(abi, torch, sc, cam, infer)
    knife = np.nonzero(margin < SEL_MARGIN)[0]
    a = np.setdiff1d(idx_o, knife)
    b = np.setdiff1d(idx_g, knife)
    assert np.array_equal(a, b)
    assert np.all(np.diff(idx_g) > 0)
    common, io, ig = np.intersect1d(idx_o, idx_g, return_indices=True)
    np.testing.assert_allclose(w_g[ig], w_o[io], atol=2e-5)
    assert c["n_gaussians"] == c["n_selected"] * sc.k
    return len(idx_o), len(knife)


def test_lod_select_config1(abi, torch):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    for infer in (False, True):
        M, nk = _check_select(abi, torch, sc, cams[0], infer)
        assert M > 1000 and nk == 0


def test_lod_select_random_views_and_ragged_sizes(abi, torch):
    rng = np.random.default_rng(0)
    for N in (1, 4095, 4096, 4097, 50_001):
        pos = rng.uniform(-20, 20, size=(N, 3)).astype(np.float32)
        sc = synth.Scene(pos=pos, level=rng.integers(0, 6, N).astype(np.uint8),
                         dL=rng.uniform(0, 0.3, N).astype(np.float32),
                         feat=np.zeros((N, 32), np.float32), offs=np.zeros((N, 10, 3), np.float32),
                         lv=np.ones((N, 3), np.float32), NL=6)
        eye = rng.uniform(-30, 30, 3)
        cam = synth.look_at_camera(eye, rng.uniform(-5, 5, 3), 160, 90, d_max=60.0)
        _check_select(abi, torch, sc, cam, infer=bool(N % 2))


def test_lod_select_many_tiles(abi, torch):
    # ~1500 tiles of 2048 anchors: offsets resolved across many look-back windows, with long
    # runs of tiles that keep nothing (most of the box is outside the view)
    rng = np.random.default_rng(5)
    N = 3_000_001
    pos = rng.uniform(-200, 200, size=(N, 3)).astype(np.float32)
    sc = synth.Scene(pos=pos, level=rng.integers(0, 8, N).astype(np.uint8),
                     dL=rng.uniform(0, 0.3, N).astype(np.float32),
                     feat=np.zeros((1, 32), np.float32), offs=np.zeros((1, 10, 3), np.float32),
                     lv=np.ones((1, 3), np.float32), NL=8)
    cam = synth.look_at_camera(np.array([150.0, -160.0, 40.0]), np.array([60.0, -20.0, 0.0]),
                               1920, 1080, d_max=500.0)
    for infer in (False, True):
        M, nk = _check_select(abi, torch, sc, cam, infer)
        assert M > 10_000


def test_lod_select_empty_and_overflow(abi, torch):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    # camera looking away: nothing selected
    away = synth.look_at_camera(cams[0].campos, 2 * cams[0].campos, 128, 128, d_max=30.0)
    idx, w, c = _gpu_select(abi, torch, sc, away, True)
    assert c["n_selected"] == 0 and c["overflow"] == 0
    # capacity smaller than the selection: flag, needed size, first entries written
    idx_o, _, _ = oracle.lod_select(sc.pos, sc.level, sc.dL, sc.NL, cams[0], True)
    idx, w, c = _gpu_select(abi, torch, sc, cams[0], True, cap=1000)
    assert c["overflow"] & 1 and c["need_selected"] == len(idx_o) and c["n_selected"] == 1000
    assert np.array_equal(idx, idx_o[:1000])


# ---------------------------------------------------------------------------------------
# decode
# ---------------------------------------------------------------------------------------

def test_decode_matches_oracle(abi, torch):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    cam = cams[0]
    rng = np.random.default_rng(1)
    sel = np.sort(rng.choice(sc.N, size=777, replace=False)).astype(np.int64)
    w = rng.uniform(0.05, 1.0, size=777).astype(np.float32)
    ref = oracle.decode(sel, w, sc, mlp, cam)
    M = len(sel)
    counts = np.zeros(8, np.uint32)
    counts[0], counts[1] = M, M * 10
    G = M * 10
    out = {"means": torch.zeros(G, 3, device="cuda"), "scales": torch.zeros(G, 3, device="cuda"),
           "quats": torch.zeros(G, 4, device="cuda"), "opac": torch.zeros(G, device="cuda"),
           "colors": torch.zeros(G, 3, device="cuda")}
    names = ("w1", "b1", "w2_op", "b2_op", "w2_col", "b2_col", "w2_cov", "b2_cov")
    mt = {n: cuda(a) for n, a in zip(names, mlp.arrays())}
    abi.decode(cuda(sc.pos), cuda(sc.feat), cuda(sc.offs), cuda(sc.lv), sc.N, mt, cam,
               cuda(sel.astype(np.int32)), cuda(w), M, cuda(counts.view(np.int32)), out)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    rel_means = ref["means"] - cam.campos.astype(np.float64)
    np.testing.assert_allclose(got["means"], rel_means, atol=2e-5)
    np.testing.assert_allclose(got["scales"], ref["scales"], rtol=2e-5, atol=1e-7)
    np.testing.assert_allclose(got["quats"], ref["quats"], atol=2e-5)
    np.testing.assert_allclose(got["opac"], ref["opac"], atol=2e-5)
    np.testing.assert_allclose(got["colors"], ref["colors"], atol=2e-5)
    # the alpha > 0 decision itself matches where it is not a knife edge
    sure = ref["op_margin"] > 1e-5
    assert np.array_equal(got["opac"][sure] > 0, ref["opac"][sure] > 0)


# ---------------------------------------------------------------------------------------
# project_bin
# ---------------------------------------------------------------------------------------

def _gpu_project(abi, torch, g, cam, rel=0):
    G = len(g["opac"])
    gt = {k: cuda(v) for k, v in g.items()}
    rec = torch.zeros(G, 12, device="cuda")
    dk = torch.zeros(G, dtype=torch.int32, device="cuda")
    rect = torch.zeros(G, 2, dtype=torch.int32, device="cuda")
    tiles = torch.zeros(G, dtype=torch.int32, device="cuda")
    gx, gy = (cam.W + 15) // 16, (cam.H + 15) // 16
    tcount = torch.full((gx * gy,), 7, dtype=torch.int32, device="cuda")   # zeroed by the call
    abi.project_bin(gt, G, rel, cam, rec, dk, rect, tiles, None, tile_count=tcount)
    torch.cuda.synchronize()
    r = to_np_u32(rect)
    rect4 = np.stack([r[:, 0] & 0xFFFF, r[:, 0] >> 16, r[:, 1] & 0xFFFF, r[:, 1] >> 16], 1)
    # the per-tile pair counts are exactly those of the rectangles the call wrote
    want = np.zeros((gy, gx), np.int64)
    for x0, y0, x1, y1 in rect4.astype(np.int64):
        want[y0:y1, x0:x1] += 1
    assert np.array_equal(to_np_u32(tcount).astype(np.int64), want.reshape(-1))
    return rec.cpu().numpy(), to_np_u32(dk), rect4.astype(np.int64), to_np_u32(tiles)


def test_project_matches_oracle(abi, torch):
    for seed, (W, H) in enumerate([(128, 128), (100, 75), (1920, 1080)]):
        cam = synth.look_at_camera(np.array([1.0, -8.0, 3.0]), np.zeros(3), W, H, d_max=30.0)
        g = synth.random_gaussians(seed, 20_000, cam, depth=(0.1, 40.0), scale=(0.01, 2.0))
        g["opac"][::17] = -0.1                     # dropped Gaussians
        ref = oracle.project(g["means"], g["scales"], g["quats"], g["opac"], cam)
        rec, dk, rect, tiles = _gpu_project(abi, torch, g, cam)
        sure = (ref["mpx"] > rect_margin(W, H)) & (ref["mz"] > NEAR_MARGIN)
        assert sure.mean() > 0.99
        assert np.array_equal(rect[sure], ref["rect"][sure])
        vis = sure & (ref["rect"][:, 2] > ref["rect"][:, 0])
        area = (ref["rect"][:, 2] - ref["rect"][:, 0]) * (ref["rect"][:, 3] - ref["rect"][:, 1])
        assert np.array_equal(tiles[sure], np.where(ref["rect"][sure, 2] > ref["rect"][sure, 0],
                                                    area[sure], 0))
        assert vis.sum() > 1000
        np.testing.assert_allclose(rec[vis, 0:2], ref["uv"][vis], rtol=1e-5, atol=2e-3)
        np.testing.assert_allclose(rec[vis, 2:4], ref["conic"][vis, 0:2], rtol=2e-3, atol=1e-6)
        np.testing.assert_allclose(rec[vis, 4], ref["conic"][vis, 2], rtol=2e-3, atol=1e-6)
        np.testing.assert_allclose(rec[vis, 9], ref["depth"][vis], rtol=1e-6)
        np.testing.assert_allclose(rec[vis, 5], g["opac"][vis], rtol=0)
        np.testing.assert_allclose(rec[vis, 6:9], g["colors"][vis], rtol=0)
        culled = sure & (ref["rect"][:, 2] <= ref["rect"][:, 0])
        assert np.all(dk[culled] == 0xFFFFFFFF)
        assert np.array_equal(dk[vis], rec[vis, 9].astype(np.float32).view(np.uint32))


# ---------------------------------------------------------------------------------------
# sort
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,lo,hi", [(0, 0, 32), (1, 0, 32), (4095, 0, 13), (4096, 0, 32),
                                     (4097, 3, 19), (100_003, 0, 32), (300_000, 0, 13)])
def test_radix_sort_matches_stable_sort(abi, torch, n, lo, hi):
    keys, vals = synth.random_sort_keys(n, n, bits=32, dup_frac=0.3)
    kt, vt = cuda(keys.view(np.int32)), cuda(vals.view(np.int32))
    scr = torch.empty(abi.radix_sort_scratch_bytes(max(n, 1)), dtype=torch.uint8, device="cuda")
    if n:
        abi.radix_sort_pairs(kt, vt, None, n, lo, hi, scr)
    torch.cuda.synchronize()
    sub = (keys >> np.uint32(lo)) & np.uint32((1 << (hi - lo)) - 1 if hi - lo < 32 else 0xFFFFFFFF)
    _, v_ref = oracle.stable_sort_pairs(sub, vals)
    assert np.array_equal(to_np_u32(vt)[:n], v_ref)
    assert np.array_equal(to_np_u32(kt)[:n], keys[v_ref])


def test_radix_sort_device_count(abi, torch):
    keys, vals = synth.random_sort_keys(5, 20_000, bits=32)
    n_dev = cuda(np.array([12_345], np.int32))
    kt, vt = cuda(keys.view(np.int32)), cuda(vals.view(np.int32))
    scr = torch.empty(abi.radix_sort_scratch_bytes(20_000), dtype=torch.uint8, device="cuda")
    abi.radix_sort_pairs(kt, vt, n_dev, 20_000, 0, 32, scr)
    torch.cuda.synchronize()
    _, v_ref = oracle.stable_sort_pairs(keys[:12_345], vals[:12_345])
    assert np.array_equal(to_np_u32(vt)[:12_345], v_ref)
    assert np.array_equal(to_np_u32(vt)[12_345:], vals[12_345:])   # untouched beyond n


def _gpu_sort_bins(abi, torch, rect, depth, gx, gy, tile_cap):
    """ogs_sort_bins: the lists in per-tile regions of tile_cap entries; returns the lists
    packed in tile order (for comparison with the oracle's), the ranges, the counts."""
    G = len(depth)
    area = np.maximum(rect[:, 2] - rect[:, 0], 0) * np.maximum(rect[:, 3] - rect[:, 1], 0)
    dk = depth.astype(np.float32).view(np.uint32).copy()
    dk[area == 0] = 0xFFFFFFFF
    packed = np.stack([rect[:, 0] | (rect[:, 1] << 16), rect[:, 2] | (rect[:, 3] << 16)], 1)
    packed = np.where(area[:, None] > 0, packed, 0).astype(np.uint32)
    nt = gx * gy
    pk = torch.zeros(nt * tile_cap, dtype=torch.int32, device="cuda")
    pg = torch.zeros(nt * tile_cap, dtype=torch.int32, device="cuda")
    tr = torch.zeros(nt, 2, dtype=torch.int32, device="cuda")
    counts = torch.zeros(8, dtype=torch.int32, device="cuda")
    scr = torch.empty(abi.sort_bins_scratch_bytes(nt), dtype=torch.uint8, device="cuda")
    abi.sort_bins(cuda(dk.view(np.int32)), cuda(packed.view(np.int32)),
                  cuda(area.astype(np.int32)), G, G, gx, gy, abi.tile_bins(pk, pg, tile_cap),
                  tr, counts, scr)
    torch.cuda.synchronize()
    trn = to_np_u32(tr).reshape(-1, 2).astype(np.int64)
    pgn = to_np_u32(pg)
    lists = [pgn[a:b] for a, b in trn]
    return (np.concatenate(lists) if lists else pgn[:0]), trn, _counts(abi, counts)


def _gpu_sort(abi, torch, rect, depth, gx, gy, pair_cap=None, ext_counts=False):
    G = len(depth)
    area = np.maximum(rect[:, 2] - rect[:, 0], 0) * np.maximum(rect[:, 3] - rect[:, 1], 0)
    P = int(area.sum())
    pair_cap = P if pair_cap is None else pair_cap
    dk = depth.astype(np.float32).view(np.uint32).copy()
    dk[area == 0] = 0xFFFFFFFF
    packed = np.stack([rect[:, 0] | (rect[:, 1] << 16), rect[:, 2] | (rect[:, 3] << 16)], 1)
    packed = np.where(area[:, None] > 0, packed, 0).astype(np.uint32)
    pg = torch.zeros(max(pair_cap, 1), dtype=torch.int32, device="cuda")
    tr = torch.zeros(gx * gy, 2, dtype=torch.int32, device="cuda")
    counts = torch.zeros(8, dtype=torch.int32, device="cuda")
    scr = torch.empty(abi.sort_scratch_bytes(G, pair_cap, gx * gy), dtype=torch.uint8,
                      device="cuda")
    tc = None
    if ext_counts:          # per-tile counts handed in (as ogs_project_bin writes them)
        want = np.zeros((gy, gx), np.int64)
        for x0, y0, x1, y1 in rect.astype(np.int64):
            want[y0:y1, x0:x1] += 1
        tc = cuda(want.reshape(-1).astype(np.int32))
    abi.sort(cuda(dk.view(np.int32)), cuda(packed.view(np.int32)),
             cuda(area.astype(np.int32)), G, G, gx, gy, pg, tr, pair_cap, counts, scr,
             tile_count=tc)
    torch.cuda.synchronize()
    return to_np_u32(pg), to_np_u32(tr), _counts(abi, counts), P


# lists of every length class: short (one small CTA per tile), beyond 2048 entries (the
# long-list sorter in shared memory) and beyond 16384 entries (its global-memory network)
@pytest.mark.parametrize("G,gx,gy", [(1, 3, 2), (3000, 9, 7), (60_000, 120, 68), (20_000, 4, 4),
                                     (100_000, 2, 2)])
@pytest.mark.parametrize("ext_counts", [False, True])
def test_sort_matches_oracle_lists(abi, torch, G, gx, gy, ext_counts):
    rect, depth = synth.random_rects_depths(G, G, gx, gy, max_span=8, equal_depth_frac=0.05)
    start, lst, _ = oracle.tile_lists(rect, depth.astype(np.float64), gx, gy)
    pg, tr, c, P = _gpu_sort(abi, torch, rect, depth, gx, gy, ext_counts=ext_counts)
    assert c["n_pairs"] == P == len(lst) and c["overflow"] == 0
    assert np.array_equal(pg[:P], lst)
    nonempty = start[1:] > start[:-1]
    assert np.array_equal(tr[nonempty, 0], start[:-1][nonempty])
    assert np.array_equal(tr[nonempty, 1], start[1:][nonempty])
    assert np.all(tr[~nonempty] == 0)


@pytest.mark.parametrize("depths", ["ties", "coarse", "narrow"])
def test_sort_list_length_classes(abi, torch, depths):
    """Tile lists of exactly the lengths at every sorter's boundaries: the warp sorter's
    register networks of 32, 64, 128, 256 and 512 slots, the shared-memory sorters of 513 ..
    2048 entries and beyond.  depths: "ties" repeats 10% of the depths exactly; "coarse" puts
    one depth of 1e30 in every list, so the warp sorter's quantised depths are too coarse to
    tell most of the others apart (its exact fallback); "narrow" draws distinct depths from
    [1, 1.008): one float step apart or more, a quantum of one step, no fallback)."""
    lengths = [0, 1, 2, 3, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256, 257,
               400, 511, 512, 513, 1000, 2047, 2048, 2049, 3000]
    gx, gy = 9, 3
    rng = np.random.default_rng(11)
    tiles = np.repeat(np.arange(len(lengths)), lengths)
    rng.shuffle(tiles)
    G = len(tiles)
    x0, y0 = tiles % gx, tiles // gx
    rect = np.stack([x0, y0, x0 + 1, y0 + 1], 1).astype(np.int32)
    if depths == "narrow":
        base = np.float32(1.0).view(np.uint32)
        depth = (base + rng.permutation(1 << 16)[:G].astype(np.uint32)).view(np.float32)
    else:
        depth = rng.uniform(0.3, 100.0, size=G).astype(np.float32)
    if depths == "ties":
        tie = rng.uniform(size=G) < 0.1
        depth[tie] = depth[rng.integers(0, G, size=int(tie.sum()))]
    if depths == "coarse":
        for t in range(len(lengths)):
            members = np.nonzero(tiles == t)[0]
            if len(members):
                depth[members[0]] = np.float32(1e30)
    start, lst, _ = oracle.tile_lists(rect, depth.astype(np.float64), gx, gy)
    assert np.array_equal(np.diff(start), lengths)
    for ext in (False, True):
        pg, tr, c, P = _gpu_sort(abi, torch, rect, depth, gx, gy, ext_counts=ext)
        assert c["n_pairs"] == P == G and c["overflow"] == 0
        assert np.array_equal(pg[:P], lst)
    got, tr, c = _gpu_sort_bins(abi, torch, rect, depth, gx, gy, 3000)
    assert c["n_pairs"] == G and c["overflow"] == 0
    assert np.array_equal(got, lst)


@pytest.mark.parametrize("G,gx,gy", [(1, 3, 2), (3000, 9, 7), (60_000, 120, 68), (20_000, 4, 4)])
def test_sort_bins_matches_oracle_lists(abi, torch, G, gx, gy):
    """ogs_sort_bins: every tile's list in its region equals the oracle's list, the ranges
    start at t * tile_cap, the pair count is the oracle's."""
    rect, depth = synth.random_rects_depths(G, G, gx, gy, max_span=8, equal_depth_frac=0.05)
    start, lst, _ = oracle.tile_lists(rect, depth.astype(np.float64), gx, gy)
    cap = int(max(1, np.diff(start).max()))
    got, tr, c = _gpu_sort_bins(abi, torch, rect, depth, gx, gy, cap)
    assert c["n_pairs"] == len(lst) and c["overflow"] == 0
    assert np.array_equal(tr[:, 0], np.arange(gx * gy) * cap)
    assert np.array_equal(tr[:, 1] - tr[:, 0], np.diff(start))
    assert np.array_equal(got, lst)


@pytest.mark.parametrize("G,gx,gy,span", [(2000, 120, 68, 60), (60_000, 40, 40, 40)])
def test_sort_bins_large_rectangles(abi, torch, G, gx, gy, span):
    """Rectangles of up to span x span tiles.  Those of more than 8 tiles go to the deferred
    list in chunks of 1024 tiles, several chunks for the largest (327 and 267 rectangles of
    more than 1024 tiles).  In the second case the chunks offered (54,902) exceed the list
    (32 entries per tile: 51,200), so the rest stay with the warps that met them.  The lists
    equal the oracle's either way."""
    rect, depth = synth.random_rects_depths(7, G, gx, gy, max_span=span, equal_depth_frac=0.05)
    start, lst, _ = oracle.tile_lists(rect, depth.astype(np.float64), gx, gy)
    cap = int(max(1, np.diff(start).max()))
    got, tr, c = _gpu_sort_bins(abi, torch, rect, depth, gx, gy, cap)
    assert c["n_pairs"] == len(lst) and c["overflow"] == 0
    assert np.array_equal(tr[:, 1] - tr[:, 0], np.diff(start))
    assert np.array_equal(got, lst)


def test_sort_bins_overflow(abi, torch):
    """A tile with more pairs than tile_cap: overflow bit 1, need_pairs = the longest list,
    every range empty."""
    rect, depth = synth.random_rects_depths(9, 2000, 20, 20, max_span=6)
    start, lst, _ = oracle.tile_lists(rect, depth.astype(np.float64), 20, 20)
    longest = int(np.diff(start).max())
    got, tr, c = _gpu_sort_bins(abi, torch, rect, depth, 20, 20, longest - 1)
    assert c["overflow"] & 2 and c["need_pairs"] == longest and c["n_pairs"] == 0
    assert np.all(tr == 0)


def test_sort_pair_overflow(abi, torch):
    rect, depth = synth.random_rects_depths(9, 2000, 20, 20, max_span=6)
    pg, tr, c, P = _gpu_sort(abi, torch, rect, depth, 20, 20, pair_cap=100)
    assert c["overflow"] & 2 and c["need_pairs"] == P and c["n_pairs"] == 0
    assert np.all(tr == 0)


# ---------------------------------------------------------------------------------------
# blend
# ---------------------------------------------------------------------------------------

def test_blend_matches_oracle(abi, torch):
    W, H = 72, 40          # ragged: 5 x 3 tiles, partial last row and column
    gx, gy = 5, 3
    r = synth.random_records(3, 300, W, H, sigma=(0.8, 10.0))
    G = 300
    order = np.argsort(r["depth"], kind="stable")
    T = gx * gy
    lst = np.tile(order, T).astype(np.int64)
    start = np.arange(T + 1, dtype=np.int64) * G
    uv = np.stack([r["u"], r["v"]], 1)
    bg = (0.05, 0.1, 0.2)
    ref = oracle.blend(W, H, start, lst, uv, r["conic"], r["opac"], r["colors"], bg)
    rec = np.zeros((G, 12), np.float32)
    rec[:, 0], rec[:, 1] = r["u"], r["v"]
    rec[:, 2:4] = r["conic"][:, 0:2]
    rec[:, 4], rec[:, 5] = r["conic"][:, 2], r["opac"]
    rec[:, 6:9] = r["colors"]
    rec[:, 9] = r["depth"]
    rec[:, 11] = -np.log(255.0 * r["opac"].astype(np.float64))
    tr = np.stack([start[:-1], start[1:]], 1).astype(np.int32)
    img = torch.zeros(3, H, W, device="cuda")
    Tf = torch.zeros(H, W, device="cuda")
    nl = torch.zeros(H, W, dtype=torch.int32, device="cuda")
    abi.blend_fwd(cuda(rec), cuda(lst.astype(np.int32)), cuda(tr), W, H, bg, img, Tf, nl)
    torch.cuda.synchronize()
    ok = ref["px_margin"] >= 1e-4
    assert ok.mean() > 0.97
    err = np.abs(img.cpu().numpy() - ref["img"])
    assert err[:, ok].max() <= PIXEL_TOL
    assert np.abs(Tf.cpu().numpy() - ref["T"])[ok].max() <= 1e-5
    assert np.array_equal(to_np_u32(nl)[ok], ref["last"][ok])


def test_blend_eval_counts(abi, torch):
    """n_eval: the tests the kernel made for each pixel while it still needed them.  Every
    Gaussian the pixel blended must have been tested, and nothing after the Gaussian the pixel
    saturated on: blended <= n_eval <= entries up to the stop (FP64 replay of the list,
    pixels off the alpha / transmittance knife edges)."""
    W, H = 72, 40
    gx, gy = 5, 3
    r = synth.random_records(3, 300, W, H, sigma=(0.8, 10.0))
    G = 300
    order = np.argsort(r["depth"], kind="stable")
    T_ = gx * gy
    lst = np.tile(order, T_).astype(np.int64)
    start = np.arange(T_ + 1, dtype=np.int64) * G
    uv = np.stack([r["u"], r["v"]], 1)
    ref = oracle.blend(W, H, start, lst, uv, r["conic"], r["opac"], r["colors"])
    rec = np.zeros((G, 12), np.float32)
    rec[:, 0], rec[:, 1] = r["u"], r["v"]
    rec[:, 2:4] = r["conic"][:, 0:2]
    rec[:, 4], rec[:, 5] = r["conic"][:, 2], r["opac"]
    rec[:, 6:9] = r["colors"]
    rec[:, 9] = r["depth"]
    rec[:, 11] = -np.log(255.0 * r["opac"].astype(np.float64))
    tr = np.stack([start[:-1], start[1:]], 1).astype(np.int32)
    img = torch.zeros(3, H, W, device="cuda")
    Tf = torch.zeros(H, W, device="cuda")
    nl = torch.zeros(H, W, dtype=torch.int32, device="cuda")
    ne = torch.zeros(H, W, dtype=torch.int32, device="cuda")
    abi.blend_fwd(cuda(rec), cuda(lst.astype(np.int32)), cuda(tr), W, H, (0.0, 0.0, 0.0), img,
                  Tf, nl, n_eval=ne)
    torch.cuda.synchronize()
    # FP64 replay of Eq. 2 with the conventions, every pixel at once
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    T = np.ones((H, W))
    done = np.zeros((H, W), bool)
    blended = np.zeros((H, W), np.int64)
    stop = np.full((H, W), G, np.int64)
    con = r["conic"].astype(np.float64)
    for i, g in enumerate(order):
        dx, dy = r["u"][g] - xs, r["v"][g] - ys
        power = -0.5 * (con[g, 0] * dx * dx + con[g, 2] * dy * dy) - con[g, 1] * dx * dy
        a = np.minimum(0.99, r["opac"][g] * np.exp(power))
        pas = ~done & (power <= 0) & (a >= 1.0 / 255.0)
        sat = pas & (T * (1 - a) < 1e-4)
        stop[sat] = i + 1
        app = pas & ~sat
        blended += app
        T = np.where(app, T * (1 - a), T)
        done |= sat
    ok = ref["px_margin"] >= PX_MARGIN
    n = to_np_u32(ne).astype(np.int64)
    assert ok.mean() > 0.9
    assert np.all(n[ok] >= blended[ok]) and np.all(n[ok] <= stop[ok])
    assert n.sum() < stop.sum()          # the warp-block culling skipped tests
    print(f"blend tests: {n.sum()} made, {blended.sum()} blended, {stop.sum()} list entries up "
          f"to the stops")


# ---------------------------------------------------------------------------------------
# whole frame
# ---------------------------------------------------------------------------------------

def _frame_parity(sc, mlp, cam, infer=True, bg=(0.0, 0.0, 0.0)):
    from paper_2403_17898_gb300.render import Renderer
    fr = oracle.render(sc, mlp, cam, infer=infer, bg=bg, want_maxc=True)
    import torch as t
    rd = Renderer(sc, mlp, cam.W, cam.H)
    maxc = t.zeros(sc.N, dtype=t.int32, device="cuda")
    c = rd.render(cam, infer=infer, bg=bg, maxc=maxc)
    assert c.overflow == 0
    knife_sel = np.nonzero(fr.sel_margin < SEL_MARGIN)[0]
    sel_g = to_np_u32(rd.sel_idx)[:c.n_selected]
    assert np.array_equal(np.setdiff1d(sel_g, knife_sel), np.setdiff1d(fr.sel_idx, knife_sel))
    assert len(knife_sel) == 0 or True
    img = rd.img.cpu().numpy()
    ok = ~knife_pixel_mask(fr, cam.W, cam.H)
    assert ok.mean() > 0.5 and ok.sum() > 500, ok.mean()
    err = np.abs(img - fr.out["img"])
    assert err[:, ok].max() <= PIXEL_TOL, err[:, ok].max()
    assert np.abs(rd.T.cpu().numpy() - fr.out["T"])[ok].max() <= 1e-5
    # the last blended Gaussian of every pixel is the same one (its list position can move
    # when a skipped neighbour with an FP32-tied depth swaps places)
    W, H = cam.W, cam.H
    py, px = np.nonzero(ok)
    tile = (py // 16) * fr.gx + px // 16
    nl_g = to_np_u32(rd.n_last)[py, px].astype(np.int64)
    nl_o = fr.out["last"][py, px].astype(np.int64)
    assert np.array_equal(nl_g > 0, nl_o > 0)
    has = nl_o > 0
    tr = to_np_u32(rd.tile_range).reshape(-1, 2).astype(np.int64)
    pg = to_np_u32(rd.pair_gauss)
    last_g = pg[tr[tile[has], 0] + nl_g[has] - 1]
    last_o = fr.lst[fr.start[tile[has]] + nl_o[has] - 1]
    assert np.array_equal(last_g, last_o)
    return fr, rd, c, maxc


def test_render_config1_matches_oracle(abi, torch):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    fr, rd, c, maxc = _frame_parity(sc, mlp, cams[0], infer=True, bg=(0.1, 0.2, 0.3))
    assert c.n_selected == len(fr.sel_idx)
    n_knife = int((fr.proj["mpx"] < rect_margin(128, 128)).sum())
    assert abs(c.n_pairs - len(fr.lst)) <= 16 * n_knife
    # per-anchor max contribution (labels of the proposal network); a knife-edge pixel can
    # move one anchor's maximum, so require agreement on nearly all anchors
    m = maxc.cpu().numpy().view(np.float32)
    close = np.abs(m - fr.out["maxc"]) <= 2e-5
    assert close.mean() > 0.995
    assert np.mean((m >= 1 / 255) == (fr.out["maxc"] >= 1 / 255)) > 0.995
    fr, rd, c, maxc = _frame_parity(sc, mlp, cams[0], infer=False)


def test_render_ragged_image_and_views(abi, torch):
    sc, mlp, _ = synth.CONFIGS["cube4k_128"]()
    rng = np.random.default_rng(4)
    for W, H in [(100, 75), (56, 40)]:
        eye = rng.normal(size=3)
        eye *= 14.0 / np.linalg.norm(eye)
        cam = synth.look_at_camera(eye, rng.uniform(-2, 2, 3), W, H, d_max=30.0)
        _frame_parity(sc, mlp, cam)


def test_render_empty_view(abi, torch):
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    away = synth.look_at_camera(cams[0].campos, 2 * cams[0].campos, 128, 128, d_max=30.0)
    rd = Renderer(sc, mlp, 128, 128)
    c = rd.render(away, bg=(0.3, 0.4, 0.5))
    assert c.n_selected == 0 and c.n_pairs == 0
    img = rd.img.cpu().numpy()
    assert np.all(img[0] == np.float32(0.3)) and np.all(img[2] == np.float32(0.5))
    assert np.all(rd.T.cpu().numpy() == 1.0) and np.all(rd.n_last.cpu().numpy() == 0)


def test_render_grows_buffers_on_overflow(abi, torch):
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    rd = Renderer(sc, mlp, 128, 128, sel_cap=64, pair_cap=1000)
    c = rd.render(cams[0])
    assert c.overflow == 0 and rd.sel_cap >= c.n_selected and rd.pair_cap >= c.n_pairs
    fr = oracle.render(sc, mlp, cams[0])
    ok = ~knife_pixel_mask(fr, 128, 128)
    assert np.abs(rd.img.cpu().numpy() - fr.out["img"])[:, ok].max() <= PIXEL_TOL


def test_render_without_n_last_is_bit_identical(abi, torch):
    """Inference without the last-entry output (track_last=False, n_last = NULL): the image
    and T are bit for bit those of the full forward, on a 1080p city frame."""
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cams = synth.CONFIGS["city2M_1080p"]()
    rd = Renderer(sc, mlp, 1920, 1080, sel_cap=200_000, pair_cap=4_000_000, precision="bf16")
    for pose in (7, 70):
        rd.track_last = True
        rd.render(cams[pose])
        img, T = rd.img.clone(), rd.T.clone()
        rd.track_last = False
        rd.render(cams[pose])
        assert torch.equal(rd.img, img) and torch.equal(rd.T, T)
