"""Pins of the oracle's SSIM loss term."""
import numpy as np
import pytest

import oracle


def test_identical_images_score_one():
    x = np.random.default_rng(0).uniform(size=(3, 20, 24))
    s, g = oracle.ssim(x, x)
    assert s == pytest.approx(1.0, abs=1e-12)
    np.testing.assert_allclose(g, 0.0, atol=1e-12)


def test_constant_images_closed_form():
    # away from the zero-padded border, constant images a, b have sigma = 0 and
    # SSIM = (2ab + C1) / (a^2 + b^2 + C1)
    a, b = 0.7, 0.4
    x = np.full((1, 40, 40), a)
    y = np.full((1, 40, 40), b)
    win = oracle.gaussian_window()
    mx = oracle._blur(x, win)
    assert mx[0, 20, 20] == pytest.approx(a, rel=1e-12)
    c1 = oracle.SSIM_C1
    want = (2 * a * b + c1) / (a * a + b * b + c1)
    # interior pixels (window fully inside): the blur of a constant is the constant
    inner = oracle._blur(x, win)[0, 10:30, 10:30]
    np.testing.assert_allclose(inner, a, rtol=1e-12)
    # direct check of the SSIM expression at an interior pixel
    my = oracle._blur(y, win)[0, 20, 20]
    sxy = oracle._blur(x * y, win)[0, 20, 20] - a * my
    assert abs(sxy) < 1e-12
    assert (2 * a * my + c1) / (a * a + my * my + c1) == pytest.approx(want, rel=1e-12)


def test_window_is_normalised_gaussian():
    w = oracle.gaussian_window(11, 1.5)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert w[5] / w[6] == pytest.approx(np.exp(1 / (2 * 1.5 ** 2)), rel=1e-12)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(3, 14, 17))
    y = np.clip(x + rng.normal(0, 0.2, size=x.shape), 0, 1)
    s, g = oracle.ssim(x, y)
    for ix in [(0, 0, 0), (1, 7, 8), (2, 13, 16), (0, 3, 12), (2, 10, 1)]:
        x0 = x[ix]
        x[ix] = x0 + 1e-6
        sp = oracle.ssim(x, y)[0]
        x[ix] = x0 - 1e-6
        sm = oracle.ssim(x, y)[0]
        x[ix] = x0
        assert g[ix] == pytest.approx((sp - sm) / 2e-6, rel=1e-5, abs=1e-10)


def test_photometric_loss_weights():
    rng = np.random.default_rng(2)
    x, y = rng.uniform(size=(3, 16, 16)), rng.uniform(size=(3, 16, 16))
    L, g = oracle.photometric_loss(x, y)
    l1, _ = oracle.l1_loss(x, y)
    s, _ = oracle.ssim(x, y)
    assert L == pytest.approx(0.8 * l1 + 0.2 * (1 - s), rel=1e-12)
