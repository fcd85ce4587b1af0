"""Pins of the oracle's proposal network (inputs, forward, BCE and backward)."""
import math

import numpy as np
import pytest

import oracle
import synth


def _net(seed=0):
    return synth.ProposalMLP(*[a.astype(np.float64) for a in synth.proposal_mlp(seed=seed).arrays()])


def test_inputs_layout():
    cam = synth.look_at_camera(np.zeros(3), np.array([1.0, 0.0, 0.0]), 32, 32, d_max=40.0)
    pos = np.array([[3.0, 0.0, 4.0]])
    feat = np.arange(32, dtype=np.float64)[None, :]
    X = oracle.proposal_inputs(pos, np.array([2]), feat, 5, np.array([0]), cam)
    np.testing.assert_allclose(X[0, :32], np.arange(32))
    assert X[0, 32] == 0.5                               # level 2 of 5 -> 2/4
    # camera looks down +x with z up: right = -y, down = -z, forward = +x, so the anchor at
    # (3, 0, 4) is seen at camera-frame direction (0, -4, 3) / 5
    np.testing.assert_allclose(X[0, 33:36], [0.0, -0.8, 0.6], atol=1e-7)
    assert X[0, 36] == pytest.approx(math.log(5.0 / 40.0), rel=1e-12)


def test_bias_only_network():
    net = _net()
    for a in net.arrays():
        a[...] = 0
    net.b3[0] = math.log(3.0)                            # sigmoid -> 0.75
    X = np.random.default_rng(0).normal(size=(5, 37))
    p, _ = oracle.proposal_forward(net, X)
    np.testing.assert_allclose(p, 0.75, rtol=1e-12)
    loss, g = oracle.proposal_bce_grad(net, X, np.array([1, 1, 0, 0, 1]))
    # -(3 ln .75 + 2 ln .25)/5 and dL/db3 = mean(p - y) = (5*.75 - 3)/5
    assert loss == pytest.approx(-(3 * math.log(0.75) + 2 * math.log(0.25)) / 5, rel=1e-12)
    assert g["b3"][0] == pytest.approx((5 * 0.75 - 3) / 5, rel=1e-12)
    # positives weighted 3x: loss -(3*3 ln .75 + 2 ln .25)/5, dL/db3 = (3*3*(.75-1) + 2*.75)/5
    loss, g = oracle.proposal_bce_grad(net, X, np.array([1, 1, 0, 0, 1]), 3.0)
    assert loss == pytest.approx(-(9 * math.log(0.75) + 2 * math.log(0.25)) / 5, rel=1e-12)
    assert g["b3"][0] == pytest.approx((9 * (0.75 - 1) + 2 * 0.75) / 5, rel=1e-12)


def test_single_path_copies_input():
    net = _net()
    for a in net.arrays():
        a[...] = 0
    net.w1[0, 36] = 1.0        # hidden1_0 = relu(ln(d/d_max)) ...
    net.b1[0] = 10.0           # ... shifted positive
    net.w2[0, 0] = 1.0
    net.w3[0, 0] = 1.0
    net.b3[0] = -10.0
    X = np.zeros((3, 37))
    X[:, 36] = [-2.0, -1.0, 0.5]
    p, t = oracle.proposal_forward(net, X)
    np.testing.assert_allclose(t["z"], X[:, 36], atol=1e-12)


@pytest.mark.parametrize("pw", [1.0, 4.0])
def test_backward_matches_finite_differences(pw):
    rng = np.random.default_rng(1)
    net = _net(3)
    X = rng.normal(size=(40, 37))
    y = (rng.uniform(size=40) < 0.4).astype(np.float64)
    loss, g = oracle.proposal_bce_grad(net, X, y, pw)
    for name, ix in [("w1", (3, 7)), ("w1", (60, 36)), ("b1", (5,)), ("w2", (10, 20)),
                     ("b2", (63,)), ("w3", (0, 11)), ("b3", (0,))]:
        arr = getattr(net, name)
        x0 = arr[ix]
        arr[ix] = x0 + 1e-6
        lp = oracle.proposal_bce_grad(net, X, y, pw)[0]
        arr[ix] = x0 - 1e-6
        lm = oracle.proposal_bce_grad(net, X, y, pw)[0]
        arr[ix] = x0
        assert g[name][ix] == pytest.approx((lp - lm) / 2e-6, rel=1e-5, abs=1e-9), (name, ix)


def test_gated_render_composition():
    """The gate after the LOD rule: p* = 0 keeps every selected anchor (the plain render, bit
    for bit); a threshold above every probability keeps none (the background); a single-path
    network that copies the level input keeps exactly the selected anchors of the levels at or
    above its threshold, which equals the plain render of that sub-selection."""
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    cam = cams[0]
    plain = oracle.render(sc, mlp, cam)
    net = _net(1)
    g0 = oracle.render(sc, mlp, cam, gate=(net, 0.0))
    assert np.array_equal(g0.sel_idx, plain.sel_idx)
    assert np.array_equal(g0.out["img"], plain.out["img"])
    gnone = oracle.render(sc, mlp, cam, bg=(0.2, 0.3, 0.4), gate=(net, 1.5))
    assert len(gnone.sel_idx) == 0
    assert np.all(gnone.out["img"][0] == 0.2) and np.all(gnone.out["img"][2] == 0.4)
    # logit = 20 (L/(NL-1) - 0.75): p >= 1/2 exactly for the anchors of level 2 (of 3 levels)
    path = _net(2)
    for a in path.arrays():
        a[...] = 0
    path.w1[0, 32] = 1.0
    path.w2[0, 0] = 1.0
    path.w3[0, 0] = 20.0
    path.b3[0] = -15.0
    lv = oracle.render(sc, mlp, cam, gate=(path, 0.5))
    want = plain.sel_idx[sc.level[plain.sel_idx] == 2]
    assert len(want) > 100 and np.array_equal(lv.sel_idx, want)
    # the same anchors decoded, projected and blended as a plain render would
    w = plain.sel_w[sc.level[plain.sel_idx] == 2]
    g = oracle.decode(want, w, sc, mlp, cam)
    np.testing.assert_array_equal(lv.gauss["opac"], g["opac"])
