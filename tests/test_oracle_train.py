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


def test_adam_rows_all_and_none():
    """Touching every row is dense Adam; touching none changes nothing."""
    rng = np.random.default_rng(3)
    p, g = rng.normal(size=(7, 5)), rng.normal(size=(7, 5))
    m, v = rng.normal(size=(7, 5)) * 0.1, rng.uniform(size=(7, 5)) * 0.01
    dense = oracle.adam(p, g, m, v, 1e-2, 0.9, 0.999, 1e-8, 4)
    rows = oracle.adam_rows(p, g, m, v, np.arange(7), 1e-2, 0.9, 0.999, 1e-8, 4)
    for a, b in zip(dense, rows):
        np.testing.assert_array_equal(a, b)
    none = oracle.adam_rows(p, g, m, v, np.zeros(0, np.int64), 1e-2, 0.9, 0.999, 1e-8, 4)
    for a, b in zip((p, m, v), none):
        np.testing.assert_array_equal(a, b)


def test_adam_rows_skipped_step_by_hand():
    """Row 0 touched at steps 1 and 3 with gradient g, row 1 at every step, row 2 never.
    Row 0's moments after step 3: m = b1 (1 - b1) g + (1 - b1) g (no decay on step 2),
    v likewise with b2 and g^2; its step-3 update uses the step-3 bias corrections.  Row 2
    keeps its initial values; row 1 follows dense Adam."""
    b1, b2, lr, eps = 0.9, 0.999, 0.01, 1e-12
    g = np.array([[0.5, -2.0], [1.5, 0.25], [3.0, 3.0]])
    p0 = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])
    p, m, v = p0.copy(), np.zeros((3, 2)), np.zeros((3, 2))
    q, mq, vq = p0[1].copy(), np.zeros(2), np.zeros(2)
    for step, rows in ((1, [0, 1]), (2, [1]), (3, [0, 1])):
        p, m, v = oracle.adam_rows(p, g, m, v, np.array(rows), lr, b1, b2, eps, step)
        q, mq, vq = oracle.adam(q, g[1], mq, vq, lr, b1, b2, eps, step)
    m_hand = b1 * (1 - b1) * g[0] + (1 - b1) * g[0]
    v_hand = b2 * (1 - b2) * g[0] ** 2 + (1 - b2) * g[0] ** 2
    np.testing.assert_allclose(m[0], m_hand, rtol=1e-14)
    np.testing.assert_allclose(v[0], v_hand, rtol=1e-14)
    # the first touch moved row 0 by lr sign(g); the second by the step-3 corrected ratio
    step1 = -lr * np.sign(g[0])
    step3 = -lr * (m_hand / (1 - b1 ** 3)) / (np.sqrt(v_hand / (1 - b2 ** 3)) + eps)
    np.testing.assert_allclose(p[0], p0[0] + step1 + step3, rtol=1e-12)
    np.testing.assert_array_equal(p[2], p0[2])
    np.testing.assert_array_equal(m[2], 0.0)
    np.testing.assert_allclose(p[1], q, rtol=1e-14)
    np.testing.assert_allclose(m[1], mq, rtol=1e-14)
