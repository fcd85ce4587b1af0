"""Pins of the oracle's appearance codes (Sec. 4.4: a learnable code per anchor, fed to the
colour MLP as an additional input).

The code enters the colour decoder's first layer exactly like extra anchor features that only
the colour decoder weighs, so a decoder whose features are extended by the code (and whose
opacity and covariance decoders give those features zero weight) must produce the same
Gaussians and, in the backward, the same gradients: the extended features' gradient is the
code's gradient and the extended colour weights' gradient is the code weights' gradient.  That
route runs through the already-pinned plain decoder, not through the appearance code path.
Zero codes reduce to the plain decoder; finite differences pin the backward once more.
"""
import copy

import numpy as np

import oracle
import synth


def _setup(seed=0, n_sel=300):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    sa, ma = synth.with_appearance(sc, mlp, seed=seed)
    cam = cams[0]
    idx, w, _ = oracle.lod_select(sc.pos, sc.level, sc.dL, sc.NL, cam, True)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(len(idx), size=min(n_sel, len(idx)), replace=False))
    return sc, mlp, sa, ma, cam, idx[pick], w[pick]


def _extended(sa, ma):
    """The same decoder written with features [f_v, a_v] and no appearance input."""
    F = sa.feat.shape[1]
    A = sa.app.shape[1]
    se = copy.copy(sa)
    se.feat = np.concatenate([sa.feat, sa.app], axis=1).astype(np.float32)
    se.app = None
    me = copy.copy(ma)
    H = ma.w1.shape[1]
    w1 = np.zeros((3, H, F + A + 4), np.float32)
    w1[:, :, :F] = ma.w1[:, :, :F]
    w1[1, :, F:F + A] = ma.w1_app
    w1[:, :, F + A:] = ma.w1[:, :, F:]
    me.w1 = w1
    me.w1_app = None
    return se, me


def test_zero_codes_reduce_to_the_plain_decoder():
    sc, mlp, sa, ma, cam, idx, w = _setup()
    sa.app = np.zeros_like(sa.app)
    a = oracle.decode(idx, w, sc, mlp, cam)
    b = oracle.decode(idx, w, sa, ma, cam)
    for k in ("means", "scales", "quats", "opac", "colors"):
        assert np.array_equal(a[k], b[k]), k


def test_codes_change_only_colours():
    sc, mlp, sa, ma, cam, idx, w = _setup()
    a = oracle.decode(idx, w, sc, mlp, cam)
    b = oracle.decode(idx, w, sa, ma, cam)
    for k in ("means", "scales", "quats", "opac"):
        assert np.array_equal(a[k], b[k]), k
    assert np.abs(a["colors"] - b["colors"]).max() > 1e-3


def test_equals_decoder_with_features_extended_by_the_code():
    sc, mlp, sa, ma, cam, idx, w = _setup(seed=1)
    se, me = _extended(sa, ma)
    a = oracle.decode(idx, w, sa, ma, cam)
    b = oracle.decode(idx, w, se, me, cam)
    for k in ("means", "scales", "quats", "opac", "colors"):
        np.testing.assert_allclose(a[k], b[k], rtol=0, atol=1e-12)


def _grads(rng, G):
    return {"dmeans": rng.normal(size=(G, 3)), "dscales": rng.normal(size=(G, 3)),
            "dquats": rng.normal(size=(G, 4)), "dopac": rng.normal(size=G),
            "dcolors": rng.normal(size=(G, 3))}


def test_backward_equals_extended_decoder_backward():
    sc, mlp, sa, ma, cam, idx, w = _setup(seed=2)
    se, me = _extended(sa, ma)
    F, A = sa.feat.shape[1], sa.app.shape[1]
    g = _grads(np.random.default_rng(3), len(idx) * sa.k)
    a = oracle.decode_bwd(idx, w, sa, ma, cam, g)
    b = oracle.decode_bwd(idx, w, se, me, cam, g)
    np.testing.assert_allclose(a["dapp"], b["dfeat"][:, F:], atol=1e-12)
    np.testing.assert_allclose(a["dfeat"], b["dfeat"][:, :F], atol=1e-12)
    np.testing.assert_allclose(a["dw1_app"], b["dw1"][1, :, F:F + A], atol=1e-12)
    np.testing.assert_allclose(a["dw1"][:, :, :F], b["dw1"][:, :, :F], atol=1e-12)
    np.testing.assert_allclose(a["dw1"][:, :, F:], b["dw1"][:, :, F + A:], atol=1e-12)
    for n in ("db1", "dw2_col", "db2_col", "doffs", "dlv"):
        np.testing.assert_allclose(a[n], b[n], atol=1e-12)


def test_backward_matches_finite_differences():
    sc, mlp, sa, ma, cam, idx, w = _setup(seed=4, n_sel=40)
    g = _grads(np.random.default_rng(5), len(idx) * sa.k)
    an = oracle.decode_bwd(idx, w, sa, ma, cam, g)

    def loss(s, m):
        o = oracle.decode(idx, w, s, m, cam)
        return float(np.sum(o["colors"] * g["dcolors"]) + np.sum(o["opac"] * g["dopac"]))

    rng = np.random.default_rng(6)
    eps = 1e-4
    for _ in range(6):                       # codes of selected anchors
        j = int(idx[rng.integers(len(idx))])
        c = int(rng.integers(sa.app.shape[1]))
        sp, sm_ = copy.copy(sa), copy.copy(sa)
        sp.app = sa.app.astype(np.float64).copy(); sp.app[j, c] += eps
        sm_.app = sa.app.astype(np.float64).copy(); sm_.app[j, c] -= eps
        fd = (loss(sp, ma) - loss(sm_, ma)) / (2 * eps)
        assert abs(fd - an["dapp"][j, c]) <= 1e-6 + 1e-5 * abs(fd), (fd, an["dapp"][j, c])
    for _ in range(6):                       # code weights
        h = int(rng.integers(ma.w1_app.shape[0]))
        c = int(rng.integers(ma.w1_app.shape[1]))
        mp, mm = copy.copy(ma), copy.copy(ma)
        mp.w1_app = ma.w1_app.astype(np.float64).copy(); mp.w1_app[h, c] += eps
        mm.w1_app = ma.w1_app.astype(np.float64).copy(); mm.w1_app[h, c] -= eps
        fd = (loss(sa, mp) - loss(sa, mm)) / (2 * eps)
        assert abs(fd - an["dw1_app"][h, c]) <= 1e-6 + 1e-5 * abs(fd), (fd, an["dw1_app"][h, c])
