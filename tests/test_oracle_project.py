"""Pins of the oracle's EWA projection and tile extent (Sec. 3.1, Eq. 1, G').

Closed forms: for a camera at the origin with R = I, a Gaussian at (x, 0, z) with isotropic
scale sigma has 2D covariance sigma^2 J J^T with J = [[fx/z, 0, -fx x/z^2], [0, fy/z, 0]],
plus the 0.3 px^2 low-pass on the diagonal.
"""
import math

import numpy as np
import pytest

import oracle
import synth

W, H = 128, 96


def _cam_identity():
    # R = I: camera looks down world +z, x right, y down
    fx = 100.0
    return synth.Camera(R=np.eye(3, dtype=np.float32), campos=np.zeros(3, np.float32),
                        fx=fx, fy=fx, cx=63.5, cy=47.5, W=W, H=H, znear=0.2, d_max=10.0)


def _proj(means, scales, quats, opac=None, cam=None):
    means = np.atleast_2d(means)
    G = len(means)
    opac = np.full(G, 0.5) if opac is None else opac
    return oracle.project(means, np.atleast_2d(scales), np.atleast_2d(quats), opac,
                          cam or _cam_identity())


ID = [1.0, 0.0, 0.0, 0.0]


def test_on_axis_axis_aligned():
    z, sx, sy = 5.0, 0.2, 0.1
    p = _proj([0.0, 0.0, z], [sx, sy, 0.7], ID)
    a = (100 * sx / z) ** 2 + 0.3
    c = (100 * sy / z) ** 2 + 0.3
    np.testing.assert_allclose(p["conic"][0], [1 / a, 0.0, 1 / c], rtol=1e-12)
    np.testing.assert_allclose(p["uv"][0], [63.5, 47.5], rtol=1e-14)
    assert p["depth"][0] == z
    # lambda_max = a (a - c > 2 sqrt(0.1)), radius 3 sqrt(a)
    assert p["radius"][0] == pytest.approx(3 * math.sqrt(a), rel=1e-12)


def test_rotation_90_about_z_swaps_axes():
    z, sx, sy = 5.0, 0.2, 0.1
    q = [math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)]
    p = _proj([0.0, 0.0, z], [sx, sy, 0.7], q)
    a = (100 * sy / z) ** 2 + 0.3
    c = (100 * sx / z) ** 2 + 0.3
    np.testing.assert_allclose(p["conic"][0], [1 / a, 0.0, 1 / c], rtol=1e-12, atol=1e-15)


def test_off_axis_isotropic_closed_form():
    x, z, s = 1.5, 6.0, 0.3
    p = _proj([x, 0.0, z], [s, s, s], ID)
    a = s * s * 100 ** 2 * (1 / z ** 2 + x ** 2 / z ** 4) + 0.3
    c = s * s * 100 ** 2 / z ** 2 + 0.3
    np.testing.assert_allclose(p["conic"][0], [1 / a, 0.0, 1 / c], rtol=1e-12, atol=1e-15)
    assert p["uv"][0, 0] == pytest.approx(100 * x / z + 63.5, rel=1e-14)


def test_frustum_clamp_of_jacobian():
    # x/z = 1.0 is beyond 1.3 tan(fov/2) = 1.3 * 128/200 = 0.832, so J uses t_x = 0.832 z:
    # J00 = fx/z, J02 = -fx 0.832/z -> a = sigma^2 fx^2 (1 + 0.832^2)/z^2 + 0.3.  A large
    # Gaussian keeps a footprint on screen.
    x, z, s = 6.0, 6.0, 3.0
    p = _proj([x, 0.0, z], [s, s, s], ID)
    lim = 1.3 * W / (2 * 100.0)
    a = s * s * 100 ** 2 * (1 + lim ** 2) / z ** 2 + 0.3
    c = s * s * 100 ** 2 / z ** 2 + 0.3
    assert p["rect"][0, 2] > p["rect"][0, 0]
    np.testing.assert_allclose(p["conic"][0], [1 / a, 0.0, 1 / c], rtol=1e-6, atol=1e-15)


def test_tile_rect_hand_case():
    # on-axis isotropic Gaussian; principal point moved so that u = 100.25
    z, s = 10.0, 0.2                     # sigma_px = 100 * 0.2 / 10 = 2 -> a = c = 4.3
    cam = _cam_identity()
    cam.cx = 100.25                     # exact in float32
    p = _proj([0.0, 0.0, z], [s, s, s], ID, cam=cam)
    a = 4.0 + 0.3
    # isotropic: mid^2 - det = 0 -> lambda = a + sqrt(0.1) (the guard), r = 3 sqrt(lambda)
    r = 3 * math.sqrt(a + math.sqrt(0.1))
    u = p["uv"][0, 0]
    assert u == 100.25
    assert p["radius"][0] == pytest.approx(r, rel=1e-12)
    # pixels ceil(u - r) .. floor(u + r) = 94 .. 106 -> tiles 5 .. 6 -> [5, 7)
    assert math.ceil(u - r) == 94 and math.floor(u + r) == 106
    assert p["rect"][0, 0] == 5 and p["rect"][0, 2] == 7
    # v = 47.5: pixels 42 .. 53 -> tiles 2 .. 3 -> [2, 4)
    assert p["rect"][0, 1] == 2 and p["rect"][0, 3] == 4


def test_culling():
    means = [[0.0, 0.0, 0.1],      # in front of the camera but inside the near plane
             [0.0, 0.0, -5.0],     # behind
             [0.0, 0.0, 5.0],      # fine, but opacity <= 0
             [200.0, 0.0, 5.0],    # far off-screen (x/z = 40)
             [0.0, 0.0, 5.0]]      # visible
    opac = np.array([0.5, 0.5, 0.0, 0.5, 0.5])
    p = _proj(means, [[0.1] * 3] * 5, [ID] * 5, opac=opac)
    empty = (p["rect"][:, 2] <= p["rect"][:, 0]) | (p["rect"][:, 3] <= p["rect"][:, 1])
    assert empty.tolist() == [True, True, True, True, False]


def test_rect_edge_margin_reported():
    # lower extent edge exactly on a tile-changing value (16m - 1 = 95) has margin 0
    z, s = 10.0, 0.2
    r = 3 * math.sqrt(4.3 + math.sqrt(0.1))
    cam = _cam_identity()
    cam.cx = 95.0 + r
    p = _proj([0.0, 0.0, z], [s, s, s], ID, cam=cam)
    assert p["mpx"][0] < 1e-5           # cx is rounded to float32
    cam.cx = 95.5 + r
    p = _proj([0.0, 0.0, z], [s, s, s], ID, cam=cam)
    assert p["mpx"][0] == pytest.approx(0.5, abs=1e-5)
