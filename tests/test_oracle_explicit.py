"""Pins of the oracle's explicit-Gaussian variant (each anchor carries k explicit 3D
Gaussians in place of the neural decoders): activation closed forms, the offset rule
(Eq. offsets), the LOD weight, and finite differences of its backward."""
import numpy as np
import pytest

import oracle
import synth


def _tiny(k=2):
    N = 3
    sc = synth.Scene(pos=np.array([[0, 0, 5], [1, 2, 3], [-1, 0, 4]], np.float32),
                     level=np.zeros(N, np.uint8), dL=np.zeros(N, np.float32),
                     feat=np.zeros((N, 32), np.float32),
                     offs=np.arange(N * k * 3, dtype=np.float32).reshape(N, k, 3) * 0.1,
                     lv=np.array([[1, 2, 3], [0.5, 0.5, 0.5], [2, 1, 1]], np.float32), NL=1, k=k)
    return sc


def test_activation_closed_forms():
    sc = _tiny()
    attr = dict(log_scale=np.zeros((3, 2, 3), np.float32), quat=np.zeros((3, 2, 4), np.float32),
                opacity=np.zeros((3, 2), np.float32), color_dc=np.zeros((3, 2, 3), np.float32))
    attr["quat"][..., 0] = 2.0
    attr["color_dc"][1, 1] = [-10.0, 1.0, 0.0]
    g = oracle.explicit_gaussians(np.array([0, 1]), np.array([1.0, 0.25]), sc, attr)
    np.testing.assert_allclose(g["scales"], 1.0)
    np.testing.assert_allclose(g["quats"], np.tile([1.0, 0, 0, 0], (4, 1)))
    np.testing.assert_allclose(g["opac"], [0.5, 0.5, 0.125, 0.125])     # sigmoid(0) * w
    np.testing.assert_allclose(g["colors"][:3], 0.5)
    np.testing.assert_allclose(g["colors"][3], [0.0, 0.5 + oracle.SH_C0, 0.5])  # clamped at 0


def test_offset_rule_and_order():
    sc = _tiny()
    rng = np.random.default_rng(0)
    attr = dict(log_scale=rng.normal(size=(3, 2, 3)), quat=rng.normal(size=(3, 2, 4)),
                opacity=rng.normal(size=(3, 2)), color_dc=rng.normal(size=(3, 2, 3)))
    sel = np.array([2, 0])
    g = oracle.explicit_gaussians(sel, np.ones(2), sc, attr)
    for r, j in enumerate(sel):
        for i in range(2):
            want = sc.pos[j].astype(np.float64) + sc.offs[j, i] * sc.lv[j].astype(np.float64)
            np.testing.assert_allclose(g["means"][2 * r + i], want, rtol=1e-12)
            np.testing.assert_allclose(g["scales"][2 * r + i], np.exp(attr["log_scale"][j, i]))


def test_backward_matches_finite_differences():
    sc = _tiny()
    rng = np.random.default_rng(1)
    attr = dict(log_scale=rng.normal(0, 0.5, size=(3, 2, 3)), quat=rng.normal(size=(3, 2, 4)),
                opacity=rng.normal(size=(3, 2)), color_dc=rng.normal(size=(3, 2, 3)))
    sel, w = np.array([0, 2]), np.array([1.0, 0.6])
    G = 4
    up = dict(dmeans=rng.normal(size=(G, 3)), dscales=rng.normal(size=(G, 3)),
              dquats=rng.normal(size=(G, 4)), dopac=rng.normal(size=G),
              dcolors=rng.normal(size=(G, 3)))

    def loss(at, scene):
        g = oracle.explicit_gaussians(sel, w, scene, at)
        return sum(float((g[a] * up[b]).sum()) for a, b in
                   (("means", "dmeans"), ("scales", "dscales"), ("quats", "dquats"),
                    ("opac", "dopac"), ("colors", "dcolors")))

    ref = oracle.explicit_gaussians_bwd(sel, w, sc, attr, up)
    h = 1e-6
    for name, key in (("log_scale", "dlog_scale"), ("quat", "dquat"), ("opacity", "dopacity"),
                      ("color_dc", "dcolor_dc")):
        for idx in [(0, 1), (2, 0)]:
            inner = attr[name].shape[2:]
            for c in np.ndindex(*inner) if inner else [()]:
                pos = idx + tuple(c)
                ap = {n: v.copy() for n, v in attr.items()}
                am = {n: v.copy() for n, v in attr.items()}
                ap[name][pos] += h
                am[name][pos] -= h
                fd = (loss(ap, sc) - loss(am, sc)) / (2 * h)
                assert ref[key][pos] == pytest.approx(fd, rel=1e-6, abs=1e-8), (name, pos)
    for name, key in (("offs", "doffs"), ("lv", "dlv")):
        base = getattr(sc, name).astype(np.float64)
        for pos in [(0, 1, 2), (2, 0, 0)] if name == "offs" else [(0, 1), (2, 2)]:
            sp, sm = _tiny(), _tiny()
            getattr(sp, name)[...] = base
            getattr(sm, name)[...] = base
            vp = base.copy(); vp[pos] += 1e-3
            vm = base.copy(); vm[pos] -= 1e-3
            object.__setattr__(sp, name, vp)
            object.__setattr__(sm, name, vm)
            fd = (loss(attr, sp) - loss(attr, sm)) / 2e-3
            assert ref[key][pos] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_unselected_anchors_get_no_gradient():
    sc = _tiny()
    rng = np.random.default_rng(2)
    attr = dict(log_scale=rng.normal(size=(3, 2, 3)), quat=rng.normal(size=(3, 2, 4)),
                opacity=rng.normal(size=(3, 2)), color_dc=rng.normal(size=(3, 2, 3)))
    up = {k: rng.normal(size=s) for k, s in (("dmeans", (2, 3)), ("dscales", (2, 3)),
                                            ("dquats", (2, 4)), ("dopac", (2,)),
                                            ("dcolors", (2, 3)))}
    ref = oracle.explicit_gaussians_bwd(np.array([1]), np.array([1.0]), sc, attr, up)
    assert np.all(ref["dlog_scale"][[0, 2]] == 0) and np.all(ref["dlv"][[0, 2]] == 0)
