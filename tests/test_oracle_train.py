"""Pins of the oracle's loss and optimiser pieces used by the training path."""
import numpy as np

import oracle


def test_l1_loss_closed_form():
    img = np.array([[0.5, 0.25], [1.0, 0.0]])
    tgt = np.array([[0.25, 0.25], [0.0, 1.0]])
    loss, grad = oracle.l1_loss(img, tgt)
    assert loss == (0.25 + 0.0 + 1.0 + 1.0) / 4
    assert grad.tolist() == [[0.25, 0.0], [0.25, -0.25]]


def test_adam_first_step_is_signed_lr():
    g = np.array([3.0, -0.5, 1e-3])
    p, m, v = oracle.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 0.01, 0.9, 0.999, 1e-15, 1)
    # bias-corrected first moments are g and g^2, so the step is -lr * sign(g)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-9)


def test_adam_constant_gradient_converges_to_lr_steps():
    p, m, v = np.zeros(1), np.zeros(1), np.zeros(1)
    for t in range(1, 101):
        p, m, v = oracle.adam(p, np.array([2.0]), m, v, 0.1, 0.9, 0.999, 1e-15, t)
    # constant gradient: every bias-corrected step is exactly lr
    np.testing.assert_allclose(p, -0.1 * 100, rtol=1e-9)
