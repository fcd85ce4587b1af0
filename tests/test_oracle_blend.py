"""Pins of the oracle's front-to-back alpha blending (Sec. 3.1, Eq. 2).

Hand-built screen-space Gaussians at exact positions: a conic of 2 ln 2 puts G = 1/2 one
pixel from the centre, so every expected colour below is a plain product of chosen numbers.
"""
import math

import numpy as np
import pytest

import oracle
import synth

LN2 = math.log(2.0)


def _render_records(W, H, uv, conic, opac, colors, depth, radius=40.0, bg=(0, 0, 0)):
    """Records -> rects covering everything within `radius` px -> lists -> blend."""
    uv = np.atleast_2d(np.asarray(uv, float))
    G = len(uv)
    gx, gy = oracle.grid(W, H)
    rect = np.zeros((G, 4), np.int32)
    for g in range(G):
        u, v = uv[g]
        rect[g] = [max(0, math.ceil(u - radius) // 16), max(0, math.ceil(v - radius) // 16),
                   min(gx, math.floor(u + radius) // 16 + 1), min(gy, math.floor(v + radius) // 16 + 1)]
    start, lst, _ = oracle.tile_lists(rect, np.asarray(depth, float), gx, gy)
    out = oracle.blend(W, H, start, lst, uv, np.atleast_2d(conic), np.asarray(opac, float),
                       np.atleast_2d(colors), bg)
    return out, start, lst, rect


ISO = [2 * LN2, 0.0, 2 * LN2]


def test_single_gaussian_closed_form():
    c = [0.2, 0.5, 0.9]
    out, *_ = _render_records(16, 16, [[5.0, 7.0]], [ISO], [0.6], [c], [3.0])
    img = out["img"]
    np.testing.assert_allclose(img[:, 7, 5], 0.6 * np.array(c), rtol=1e-15)     # G = 1
    np.testing.assert_allclose(img[:, 7, 6], 0.3 * np.array(c), rtol=1e-15)     # G = 1/2
    np.testing.assert_allclose(img[:, 8, 6], 0.15 * np.array(c), rtol=1e-14)    # G = 1/4
    assert out["T"][7, 5] == pytest.approx(0.4, abs=1e-15)
    assert out["last"][7, 5] == 1
    # anisotropic conic with b: at d = (1, 1), power = -0.5 (a + c) - b
    conic = [LN2, -LN2 / 2, LN2]          # power = -0.5*2 ln2 + ln2/2 = -ln2/2
    out, *_ = _render_records(16, 16, [[5.0, 7.0]], [conic], [0.8], [c], [3.0])
    np.testing.assert_allclose(out["img"][:, 8, 6], 0.8 * 2 ** -0.5 * np.array(c), rtol=1e-14)


def test_two_gaussians_composite():
    c1, c2 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])
    # Gaussian 1 is behind (depth 5) but listed first; Gaussian 0 is in front (depth 2)
    out, *_ = _render_records(16, 16, [[5.0, 7.0], [5.0, 7.0]], [ISO, ISO], [0.6, 0.5],
                              [c1, c2], [2.0, 5.0])
    np.testing.assert_allclose(out["img"][:, 7, 5], 0.6 * c1 + 0.5 * 0.4 * c2, rtol=1e-15)
    assert out["T"][7, 5] == pytest.approx(0.4 * 0.5, abs=1e-15)
    # swap depths: order flips
    out, *_ = _render_records(16, 16, [[5.0, 7.0], [5.0, 7.0]], [ISO, ISO], [0.6, 0.5],
                              [c1, c2], [5.0, 2.0])
    np.testing.assert_allclose(out["img"][:, 7, 5], 0.5 * c2 + 0.6 * 0.5 * c1, rtol=1e-15)


def test_background():
    c = np.array([0.2, 0.5, 0.9])
    bg = np.array([0.1, 0.2, 0.3])
    out, *_ = _render_records(16, 16, [[5.0, 7.0]], [ISO], [0.6], [c], [3.0], bg=bg)
    np.testing.assert_allclose(out["img"][:, 7, 5], 0.6 * c + 0.4 * bg, rtol=1e-15)
    np.testing.assert_allclose(out["img"][:, 0, 15], bg, rtol=1e-15)   # far pixel


def test_alpha_clamp():
    out, *_ = _render_records(16, 16, [[5.0, 7.0]], [ISO], [1.0], [[1.0, 1.0, 1.0]], [3.0])
    assert out["img"][0, 7, 5] == pytest.approx(0.99, abs=1e-15)
    assert out["T"][7, 5] == pytest.approx(0.01, abs=1e-15)


def test_alpha_skip():
    # 0.003 < 1/255: skipped, pixel untouched and the list index does not count it
    out, *_ = _render_records(16, 16, [[5.0, 7.0]], [ISO], [0.003], [[1.0, 1.0, 1.0]], [3.0])
    assert out["img"][0, 7, 5] == 0.0 and out["T"][7, 5] == 1.0 and out["last"][7, 5] == 0
    # just above 1/255 contributes
    out, *_ = _render_records(16, 16, [[5.0, 7.0]], [ISO], [0.004], [[1.0, 1.0, 1.0]], [3.0])
    assert out["img"][0, 7, 5] == pytest.approx(0.004, abs=1e-15)


def test_early_stop():
    # three alpha = 0.98 Gaussians: T 1 -> 0.02 -> 4e-4; the third would give 8e-6 < 1e-4
    cols = np.eye(3)
    out, *_ = _render_records(16, 16, [[5.0, 7.0]] * 3, [ISO] * 3, [0.98] * 3, cols,
                              [1.0, 2.0, 3.0])
    np.testing.assert_allclose(out["img"][:, 7, 5], [0.98, 0.98 * 0.02, 0.0], atol=1e-15)
    assert out["T"][7, 5] == pytest.approx(4e-4, rel=1e-12)
    assert out["last"][7, 5] == 2


def test_transmittance_monotone_and_bounded():
    rng = np.random.default_rng(0)
    G = 60
    uv = rng.uniform(0, 48, size=(G, 2))
    conic = np.tile([0.05, 0.0, 0.05], (G, 1))
    opac = rng.uniform(0.05, 0.9, size=G)
    col = rng.uniform(size=(G, 3))
    depth = rng.uniform(1, 10, size=G)
    out, *_ = _render_records(48, 48, uv, conic, opac, col, depth)
    T1 = out["T"]
    assert np.all(T1 > 0) and np.all(T1 <= 1)
    # a Gaussian added in front of everything never raises T anywhere
    out2, *_ = _render_records(48, 48, np.vstack([uv, [[24.0, 24.0]]]),
                               np.vstack([conic, [[0.01, 0.0, 0.01]]]),
                               np.append(opac, 0.5), np.vstack([col, [[1, 1, 1]]]),
                               np.append(depth, 0.5))
    # early stop can leave T slightly above the product of all (1 - a_i); still never above
    assert np.all(out2["T"] <= T1 + 1e-15)


def _project_random(seed, G, W, H):
    cam = synth.look_at_camera(np.array([0.0, -6.0, 1.5]), np.zeros(3), W, H, d_max=20.0)
    g = synth.random_gaussians(seed, G, cam, depth=(2.0, 12.0), scale=(0.05, 0.6))
    pr = oracle.project(g["means"], g["scales"], g["quats"], g["opac"], cam)
    return g, pr


def test_input_order_invariance():
    W, H = 48, 32
    g, pr = _project_random(1, 40, W, H)
    gx, gy = oracle.grid(W, H)
    vis = pr["rect"][:, 2] > pr["rect"][:, 0]
    assert len(np.unique(pr["depth"][vis])) == vis.sum() > 20
    start, lst, _ = oracle.tile_lists(pr["rect"], pr["depth"], gx, gy)
    a = oracle.blend(W, H, start, lst, pr["uv"], pr["conic"], g["opac"], g["colors"])
    perm = np.random.default_rng(2).permutation(40)
    start2, lst2, _ = oracle.tile_lists(pr["rect"][perm], pr["depth"][perm], gx, gy)
    b = oracle.blend(W, H, start2, lst2, pr["uv"][perm], pr["conic"][perm], g["opac"][perm],
                     g["colors"][perm])
    assert np.array_equal(a["img"], b["img"]) and np.array_equal(a["T"], b["T"])


def test_brute_force_per_pixel():
    """Per pixel, every Gaussian whose rect covers the pixel's tile, sorted by (depth, id),
    blended one by one in plain Python: equals the tiled result."""
    W, H = 40, 24
    g, pr = _project_random(3, 30, W, H)
    gx, gy = oracle.grid(W, H)
    start, lst, _ = oracle.tile_lists(pr["rect"], pr["depth"], gx, gy)
    out = oracle.blend(W, H, start, lst, pr["uv"], pr["conic"], g["opac"], g["colors"])
    opac = g["opac"].astype(np.float64)
    col = g["colors"].astype(np.float64)
    for py in range(H):
        for px in range(W):
            tx, ty = px // 16, py // 16
            cand = [i for i in range(30) if pr["rect"][i, 0] <= tx < pr["rect"][i, 2]
                    and pr["rect"][i, 1] <= ty < pr["rect"][i, 3]]
            cand.sort(key=lambda i: (pr["depth"][i], i))
            T, C = 1.0, np.zeros(3)
            for i in cand:
                dx, dy = pr["uv"][i, 0] - px, pr["uv"][i, 1] - py
                a, b, c = pr["conic"][i]
                pw = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
                if pw > 0:
                    continue
                al = min(0.99, opac[i] * math.exp(pw))
                if al < 1 / 255:
                    continue
                if T * (1 - al) < 1e-4:
                    break
                C += col[i] * al * T
                T *= 1 - al
            np.testing.assert_allclose(out["img"][:, py, px], C, rtol=1e-12, atol=1e-15)
            assert out["T"][py, px] == pytest.approx(T, rel=1e-12, abs=1e-15)
