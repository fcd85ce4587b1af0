"""GPU photometric loss (0.8 L1 + 0.2 D-SSIM) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from gpu_helpers import cuda, lib_ready

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cached", [False, True])
@pytest.mark.parametrize("shape", [(3, 16, 16), (3, 75, 100), (3, 270, 480)])
def test_l1_ssim_matches_oracle(shape, cached):
    """Both forms: the target's window moments blurred in the loss pass, or precomputed once
    by ogs_ssim_target_stats and passed in."""
    import torch
    abi = lib_ready()
    rng = np.random.default_rng(shape[1])
    x = rng.uniform(size=shape).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.15, size=shape), 0, 1).astype(np.float32)
    L_ref, g_ref = oracle.photometric_loss(x, y, 0.2)
    dimg = torch.zeros(shape, device="cuda")
    loss = torch.zeros(1, device="cuda")
    scr = torch.empty(abi.loss_l1_ssim_scratch_bytes(*shape), dtype=torch.uint8, device="cuda")
    stats = None
    if cached:
        stats = torch.empty((2,) + shape, device="cuda")
        abi.ssim_target_stats(cuda(y), stats)
    abi.loss_l1_ssim(cuda(x), cuda(y), 0.2, dimg, loss, scr, target_stats=stats)
    torch.cuda.synchronize()
    assert abs(loss.item() - L_ref) <= 2e-5
    g = dimg.cpu().numpy()
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_ssim_target_stats_are_the_window_moments():
    """ogs_ssim_target_stats = the zero-padded 11x11 Gaussian window means of y and y^2, as the
    oracle's own separable blur computes them."""
    import torch
    abi = lib_ready()
    rng = np.random.default_rng(9)
    y = rng.uniform(size=(3, 45, 70)).astype(np.float32)
    stats = torch.empty((2,) + y.shape, device="cuda")
    abi.ssim_target_stats(cuda(y), stats)
    torch.cuda.synchronize()
    win = oracle.gaussian_window()
    got = stats.cpu().numpy()
    np.testing.assert_allclose(got[0], oracle._blur(y.astype(np.float64), win), atol=2e-6)
    np.testing.assert_allclose(got[1], oracle._blur(y.astype(np.float64) ** 2, win), atol=2e-6)
