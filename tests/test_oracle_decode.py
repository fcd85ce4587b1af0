"""Pins of the oracle's neural-Gaussian decoding (Sec. 3.2, Eq. offsets and Eq. mlp).

Each case uses weights whose output is known in closed form (inverse activations, a
single-path network that copies one input, or an all-active network that collapses to one
affine map), so a swapped input, a dropped bias or a wrong activation fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synth

K = 10
F = 32
HD = 32


def _scene(pos, feat=None, offs=None, lv=None):
    N = len(pos)
    rng = np.random.default_rng(0)
    return synth.Scene(
        pos=np.asarray(pos, np.float32),
        level=np.zeros(N, np.uint8), dL=np.zeros(N, np.float32),
        feat=(rng.normal(0, 0.1, (N, F)) if feat is None else feat).astype(np.float32),
        offs=(rng.normal(0, 0.5, (N, K, 3)) if offs is None else offs).astype(np.float32),
        lv=(np.full((N, 3), 0.5) if lv is None else lv).astype(np.float32), NL=1, k=K)


def _zero_mlp():
    z = np.zeros
    return synth.DecoderMLP(z((3, HD, F + 4), np.float32), z((3, HD), np.float32),
                            z((K, HD), np.float32), z(K, np.float32),
                            z((3 * K, HD), np.float32), z(3 * K, np.float32),
                            z((7 * K, HD), np.float32), z(7 * K, np.float32))


def _cam(campos=(0.0, 0.0, 0.0)):
    return synth.look_at_camera(np.asarray(campos, float), np.array([1.0, 0.0, 0.0]), 64, 64,
                                d_max=50.0)


def test_bias_only_closed_forms():
    mlp = _zero_mlp()
    mlp.b2_op[:] = math.atanh(0.5)             # tanh -> 0.5
    mlp.b2_col[:] = math.log(3.0)              # sigmoid -> 0.75
    cov = mlp.b2_cov.reshape(K, 7)
    cov[:, :3] = 0.0                           # sigmoid -> 0.5
    cov[:, 3:] = [3.0, 0.0, 4.0, 0.0]          # -> (0.6, 0, 0.8, 0)
    sc = _scene([[5.0, 1.0, -2.0]], lv=np.array([[2.0, 3.0, 4.0]]))
    out = oracle.decode(np.array([0]), np.array([0.4]), sc, mlp, _cam())
    np.testing.assert_allclose(out["opac"], 0.4 * 0.5, rtol=1e-6)
    np.testing.assert_allclose(out["colors"], 0.75, rtol=1e-6)
    np.testing.assert_allclose(out["scales"], np.tile([1.0, 1.5, 2.0], (K, 1)), rtol=1e-7)
    np.testing.assert_allclose(out["quats"], np.tile([0.6, 0.0, 0.8, 0.0], (K, 1)), atol=1e-7)


def test_offsets_scaled_by_lv():
    offs = np.zeros((1, K, 3))
    offs[0, :, 0] = np.arange(K)               # O_i = (i, 0, 0) ... plus a y component
    offs[0, :, 1] = -1.0
    sc = _scene([[5.0, 1.0, -2.0]], offs=offs, lv=np.array([[0.5, 2.0, 4.0]]))
    out = oracle.decode(np.array([0]), np.array([1.0]), sc, _zero_mlp(), _cam())
    expect = np.stack([5.0 + 0.5 * np.arange(K), np.full(K, 1.0 - 2.0), np.full(K, -2.0)], 1)
    np.testing.assert_allclose(out["means"], expect, atol=1e-6)


def test_input_wiring_direction_and_distance():
    """Covariance decoder copies relu(dir_x), relu(dir_y), relu(dir_z), dist into the raw
    quaternion of Gaussian 0; the anchor sits at (3, 0, 4) from the camera, so the
    quaternion is (0.6, 0, 0.8, 5)/sqrt(26)."""
    mlp = _zero_mlp()
    Din = F + 4
    for h, col in enumerate([F, F + 1, F + 2, F + 3]):
        mlp.w1[2, h, col] = 1.0
        mlp.w2_cov[3 + h, h] = 1.0
    sc = _scene([[3.0, 0.0, 4.0]])
    out = oracle.decode(np.array([0]), np.array([1.0]), sc, mlp, _cam())
    q = np.array([0.6, 0.0, 0.8, 5.0]) / math.sqrt(26.0)
    np.testing.assert_allclose(out["quats"][0], q, atol=1e-6)
    # the other Gaussians' quaternions are all-zero raw -> NaN-free check not needed; the
    # colour/opacity decoders did not see the direction
    np.testing.assert_allclose(out["colors"], 0.5, atol=1e-12)
    assert Din == 36


def test_input_wiring_feature():
    """Opacity decoder: hidden 0 = relu(f_7); opacity_3 = tanh(2 * hidden 0)."""
    mlp = _zero_mlp()
    mlp.w1[0, 0, 7] = 1.0
    mlp.w2_op[3, 0] = 2.0
    feat = np.zeros((2, F))
    feat[0, 7] = math.atanh(0.8) / 2     # -> tanh = 0.8
    feat[1, 7] = -0.3                    # relu clips -> opacity 0 -> dropped (<= 0)
    sc = _scene([[5.0, 0.0, 0.0], [6.0, 0.0, 0.0]], feat=feat)
    out = oracle.decode(np.array([0, 1]), np.array([1.0, 1.0]), sc, mlp, _cam())
    assert out["opac"][3] == pytest.approx(0.8, abs=1e-6)
    assert out["opac"][K + 3] == 0.0
    assert np.all(out["opac"][:3] == 0.0)


def test_all_active_network_is_affine():
    """With every hidden unit active (large positive b1) each decoder is the affine map
    (W2 W1) z + (W2 b1 + b2); compare logit(colour) with that collapsed map."""
    rng = np.random.default_rng(3)
    mlp = synth.decoder_mlp(seed=4, dist_scale=1.0 / 30.0)
    mlp.b1[:] = 10.0
    mlp.w2_col *= np.float32(0.05)        # keep logits O(1) so logit(colour) is well conditioned
    N = 7
    pos = rng.uniform(-5, 5, size=(N, 3)) + np.array([20.0, 0, 0])
    sc = _scene(pos)
    cam = _cam()
    out = oracle.decode(np.arange(N), np.ones(N), sc, mlp, cam)
    v = sc.pos.astype(np.float64) - cam.campos.astype(np.float64)
    d = np.linalg.norm(v, axis=1, keepdims=True)
    z = np.concatenate([sc.feat.astype(np.float64), v / d, d], 1)
    W1 = mlp.w1[1].astype(np.float64)
    W2 = mlp.w2_col.astype(np.float64)
    A = W2 @ W1
    c = W2 @ mlp.b1[1].astype(np.float64) + mlp.b2_col
    assert np.all(z @ W1.T + mlp.b1[1] > 1.0)         # every hidden unit active
    raw = z @ A.T + c                                  # [N, 3K]
    col = out["colors"].reshape(N, 3 * K)
    np.testing.assert_allclose(np.log(col / (1 - col)), raw, rtol=1e-9, atol=1e-9)


def test_transitional_weight_scales_opacity():
    sc = _scene([[8.0, 1.0, 0.0]])
    mlp = synth.decoder_mlp(seed=2)
    a = oracle.decode(np.array([0]), np.array([1.0]), sc, mlp, _cam())
    b = oracle.decode(np.array([0]), np.array([0.3]), sc, mlp, _cam())
    np.testing.assert_allclose(b["opac"], 0.3 * a["opac"], rtol=1e-14)
    np.testing.assert_allclose(b["colors"], a["colors"], rtol=0)
