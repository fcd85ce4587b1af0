"""GPU photometric loss (0.8 L1 + 0.2 D-SSIM) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from gpu_helpers import cuda, lib_ready

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(3, 16, 16), (3, 75, 100), (3, 270, 480)])
def test_l1_ssim_matches_oracle(shape):
    import torch
    abi = lib_ready()
    rng = np.random.default_rng(shape[1])
    x = rng.uniform(size=shape).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.15, size=shape), 0, 1).astype(np.float32)
    L_ref, g_ref = oracle.photometric_loss(x, y, 0.2)
    dimg = torch.zeros(shape, device="cuda")
    loss = torch.zeros(1, device="cuda")
    scr = torch.empty(abi.loss_l1_ssim_scratch_bytes(*shape), dtype=torch.uint8, device="cuda")
    abi.loss_l1_ssim(cuda(x), cuda(y), 0.2, dimg, loss, scr)
    torch.cuda.synchronize()
    assert abs(loss.item() - L_ref) <= 2e-5
    g = dimg.cpu().numpy()
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
