"""Pins of the oracle's anchor selection (Sec. 4.1.3, Eq. for L_hat, opacity blending).

Expected values are hand-derived from the equation at chosen distances, not recomputed with
the oracle's formula: an anchor at d = d_max / 2^(m + f) has fractional level m + f.
"""
import numpy as np
import pytest

import oracle
import synth

D_MAX = 64.0
NL = 5


def _axis_cam(W=64, H=64):
    # camera at the origin looking down +x (world), so distance == camera depth
    return synth.look_at_camera(np.zeros(3), np.array([1.0, 0.0, 0.0]), W, H, d_max=D_MAX)


def _on_axis(ds):
    ds = np.asarray(ds, np.float64)
    return np.stack([ds, np.zeros_like(ds), np.zeros_like(ds)], 1)


def _select(pos, level, dL=None, infer=True, cam=None, NL_=NL):
    cam = cam or _axis_cam()
    dL = np.zeros(len(pos)) if dL is None else dL
    return oracle.lod_select(pos, np.asarray(level), dL, NL_, cam, infer)


def test_fractional_level_hand_cases():
    # L* = 2.25 -> L_hat = 2: levels 0..2 full, level 3 transitional with weight 0.25
    d = D_MAX / 2 ** 2.25
    pos = _on_axis([d] * NL)
    idx, w, _ = _select(pos, np.arange(NL))
    assert idx.tolist() == [0, 1, 2, 3]
    assert w[:3].tolist() == [1.0, 1.0, 1.0]
    assert w[3] == pytest.approx(0.25, abs=1e-12)
    # training mode: no next-level anchors
    idx, w, _ = _select(pos, np.arange(NL), infer=False)
    assert idx.tolist() == [0, 1, 2] and np.all(w == 1.0)


def test_lod_bias_shifts_level():
    # d = d_max/2 -> log2 term exactly 1; dL = 0.5 -> L* = 1.5
    pos = _on_axis([D_MAX / 2] * NL)
    idx, w, _ = _select(pos, np.arange(NL), dL=np.full(NL, 0.5))
    assert idx.tolist() == [0, 1, 2]
    assert w[2] == pytest.approx(0.5, abs=1e-12)


def test_clamps():
    # very close: L* clamps at NL-1 -> every level full, nothing transitional
    pos = _on_axis([0.5] * NL)   # log2(64/0.5) = 7 > NL-1
    idx, w, _ = _select(pos, np.arange(NL))
    assert idx.tolist() == list(range(NL)) and np.all(w == 1.0)
    # very far: L* clamps at 0 -> only level 0; next-level weight would be 0 -> not selected
    pos = _on_axis([1e6] * NL)
    idx, w, _ = _select(pos, np.arange(NL))
    assert idx.tolist() == [0] and w[0] == 1.0


def test_integer_boundary_knife_edge_reported():
    # exactly at d_max/4: L* = 2, so level 2 full and level 3 has weight 0 (not selected);
    # the margin of level-2 and level-3 anchors is 0 there.
    pos = _on_axis([D_MAX / 4] * NL)
    idx, w, m = _select(pos, np.arange(NL))
    assert idx.tolist() == [0, 1, 2]
    assert m[2] == pytest.approx(0.0, abs=1e-12) and m[3] == pytest.approx(0.0, abs=1e-12)
    assert m[0] > 0.1  # level 0 is never decided by a level threshold


def test_cumulative_and_monotone_in_distance():
    rng = np.random.default_rng(5)
    ds = np.sort(rng.uniform(0.5, 200.0, size=300))
    counts_full = []
    for d in ds:
        pos = _on_axis([d] * NL)
        idx, w, _ = _select(pos, np.arange(NL))
        full = idx[w == 1.0]
        # cumulative: the fully selected levels form a prefix 0..L_hat
        assert full.tolist() == list(range(len(full)))
        # at most one transitional level, right after the prefix
        trans = idx[w < 1.0]
        assert len(trans) <= 1
        if len(trans):
            assert trans[0] == len(full) and 0.0 < w[w < 1.0][0] < 1.0
        counts_full.append(len(full))
    # farther anchors never get more levels
    assert np.all(np.diff(counts_full) <= 0)


def test_weight_is_continuous_across_levels():
    # total "level mass" sum(w) grows continuously as the camera approaches: a fine sweep's
    # largest jump shrinks with the step (opacity blending removes LOD popping)
    def mass(d):
        idx, w, _ = _select(_on_axis([d] * NL), np.arange(NL))
        return w.sum()
    for n in (200, 2000):
        ds = np.geomspace(1.0, 100.0, n)
        jumps = np.abs(np.diff([mass(d) for d in ds]))
        step = np.log2(ds[1] / ds[0])
        assert jumps.max() <= step * 1.0001 + 1e-12


def test_focal_scale_equals_scaled_distance():
    rng = np.random.default_rng(1)
    N = 2000
    cam = synth.look_at_camera(np.array([0.0, -30.0, 10.0]), np.zeros(3), 96, 64, d_max=D_MAX)
    pos = rng.uniform(-20, 20, size=(N, 3))
    level = rng.integers(0, NL, size=N)
    dL = rng.uniform(0, 0.3, size=N)
    c = cam.campos.astype(np.float64)
    cam2 = synth.Camera(**{**cam.__dict__, "s": 2.0})
    a = oracle.lod_select(pos, level, dL, NL, cam2, True)
    pos_far = c + 2.0 * (pos - c)   # exact in binary floating point
    b = oracle.lod_select(pos_far, level, dL, NL, cam, True)
    assert a[0].tolist() == b[0].tolist()
    np.testing.assert_allclose(a[1], b[1], rtol=0, atol=1e-12)


def test_visibility_test():
    cam = _axis_cam(W=64, H=64)
    tanx = cam.W / (2 * cam.fx)
    z = 10.0
    # camera looks down +x world; camera-right is world -y (right = f x up)
    inside = np.array([z, -1.29 * tanx * z, 0.0])
    outside = np.array([z, -1.31 * tanx * z, 0.0])
    behind = np.array([-z, 0.0, 0.0])
    near = np.array([0.1, 0.0, 0.0])
    pos = np.stack([inside, outside, behind, near])
    idx, w, _ = _select(pos, np.zeros(4, int))
    assert idx.tolist() == [0]


def test_selection_is_ordered_and_stable():
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    idx, w, m = oracle.lod_select(sc.pos, sc.level, sc.dL, sc.NL, cams[0], True)
    assert np.all(np.diff(idx) > 0)
    assert np.all((w > 0) & (w <= 1))
    # weights below 1 only on anchors one level above their view level
    assert len(idx) > 1000
