"""Pins of the oracle's analytic backward against central finite differences of its own
forward (FP64, step 1e-6), on tiny inputs chosen away from every decision threshold so that a
step cannot flip a skip/stop/cull decision (checked through the reported margins)."""
import numpy as np
import pytest

import oracle
import synth

H_FD = 1e-6


def _fd(f, x, idx, h=H_FD):
    x0 = x[idx]
    x[idx] = x0 + h
    fp = f()
    x[idx] = x0 - h
    fm = f()
    x[idx] = x0
    return (fp - fm) / (2 * h)


def _blend_setup(seed=0, W=32, H=32, G=24):
    cam = synth.look_at_camera(np.array([0.0, -6.0, 1.5]), np.zeros(3), W, H, d_max=20.0)
    g = synth.random_gaussians(seed, G, cam, depth=(3.0, 10.0), scale=(0.1, 0.5),
                               frac_behind=0.0)
    g["opac"] = np.minimum(g["opac"], 0.85)       # stay away from the 0.99 clamp
    pr = oracle.project(g["means"], g["scales"], g["quats"], g["opac"], cam)
    gx, gy = oracle.grid(W, H)
    start, lst, _ = oracle.tile_lists(pr["rect"], pr["depth"], gx, gy)
    rng = np.random.default_rng(seed + 100)
    dimg = rng.normal(size=(3, H, W))
    return cam, g, pr, start, lst, dimg


def test_blend_bwd_matches_fd():
    W = H = 32
    cam, g, pr, start, lst, dimg = _blend_setup()
    uv, conic = pr["uv"].copy(), pr["conic"].copy()
    opac, col = g["opac"].astype(np.float64).copy(), g["colors"].astype(np.float64).copy()
    bg = np.array([0.1, 0.3, 0.2])
    base = oracle.blend(W, H, start, lst, uv, conic, opac, col, bg)
    assert base["px_margin"].min() > 1e-5

    def f():
        return float((oracle.blend(W, H, start, lst, uv, conic, opac, col, bg)["img"] * dimg).sum())

    gb = oracle.blend_bwd(W, H, start, lst, uv, conic, opac, col, bg, dimg)
    vis = np.nonzero(pr["rect"][:, 2] > pr["rect"][:, 0])[0]
    rng = np.random.default_rng(7)
    for gidx in rng.choice(vis, size=6, replace=False):
        for arr, grad, comp in [(uv, gb["duv"], 2), (conic, gb["dconic"], 3),
                                (col, gb["dcolors"], 3)]:
            for c in range(comp):
                num = _fd(f, arr, (gidx, c))
                assert grad[gidx, c] == pytest.approx(num, rel=1e-5, abs=1e-7)
        num = _fd(f, opac, gidx)
        assert gb["dopac"][gidx] == pytest.approx(num, rel=1e-5, abs=1e-7)


def test_blend_bwd_clamped_alpha_has_no_opacity_gradient():
    # alpha = min(0.99, o G) with o G > 0.99 at the only pixel it covers meaningfully
    uv = np.array([[5.0, 7.0]])
    conic = np.array([[50.0, 0.0, 50.0]])     # tiny: neighbours get G ~ e^-25
    opac = np.array([1.0])
    col = np.array([[1.0, 0.5, 0.2]])
    rect = np.array([[0, 0, 1, 1]], np.int32)
    start, lst, _ = oracle.tile_lists(rect, np.array([1.0]), 1, 1)
    dimg = np.ones((3, 16, 16))
    gb = oracle.blend_bwd(16, 16, start, lst, uv, conic, opac, col, np.zeros(3), dimg)
    assert gb["dopac"][0] == 0.0 and np.all(gb["duv"] == 0.0)
    np.testing.assert_allclose(gb["dcolors"][0], 0.99, rtol=1e-15)


def test_project_bwd_matches_fd():
    W = H = 32
    cam, g, pr, start, lst, _ = _blend_setup(seed=2)
    means = g["means"].astype(np.float64).copy()
    scales = g["scales"].astype(np.float64).copy()
    quats = g["quats"].astype(np.float64).copy()
    opac = g["opac"].astype(np.float64)
    rng = np.random.default_rng(3)
    wuv = rng.normal(size=pr["uv"].shape)
    wcon = rng.normal(size=pr["conic"].shape) * 10

    def f():
        p = oracle.project(means, scales, quats, opac, cam)
        return float((p["uv"] * wuv).sum() + (p["conic"] * wcon).sum())

    pb = oracle.project_bwd(means, scales, quats, pr["rect"], cam, wuv, wcon)
    vis = np.nonzero(pr["rect"][:, 2] > pr["rect"][:, 0])[0]
    for gidx in vis[:6]:
        for arr, grad, comp in [(means, pb["dmeans"], 3), (scales, pb["dscales"], 3),
                                (quats, pb["dquats"], 4)]:
            for c in range(comp):
                num = _fd(f, arr, (gidx, c))
                assert grad[gidx, c] == pytest.approx(num, rel=1e-5, abs=1e-6)


def test_project_bwd_clamped_jacobian_matches_fd():
    # one large Gaussian beyond the 1.3 x half-fov bound: the clamped branch of J
    cam = synth.Camera(R=np.eye(3, dtype=np.float32), campos=np.zeros(3, np.float32),
                       fx=100.0, fy=100.0, cx=63.5, cy=47.5, W=128, H=96, znear=0.2, d_max=10.0)
    means = np.array([[6.0, -0.5, 6.0]])
    scales = np.array([[3.0, 2.0, 1.0]])
    quats = np.array([[0.9, 0.1, -0.3, 0.2]])
    quats /= np.linalg.norm(quats)
    opac = np.array([0.5])
    pr = oracle.project(means, scales, quats, opac, cam)
    assert pr["rect"][0, 2] > pr["rect"][0, 0]
    wuv = np.array([[0.3, -0.7]])
    wcon = np.array([[100.0, -50.0, 80.0]])

    def f():
        p = oracle.project(means, scales, quats, opac, cam)
        return float((p["uv"] * wuv).sum() + (p["conic"] * wcon).sum())

    pb = oracle.project_bwd(means, scales, quats, pr["rect"], cam, wuv, wcon)
    for arr, grad, comp in [(means, pb["dmeans"], 3), (scales, pb["dscales"], 3),
                            (quats, pb["dquats"], 4)]:
        for c in range(comp):
            assert grad[0, c] == pytest.approx(_fd(f, arr, (0, c)), rel=1e-5, abs=1e-8)


def _tiny_scene(seed=0, N=12):
    rng = np.random.default_rng(seed)
    sc = synth.Scene(pos=rng.uniform(-1, 1, size=(N, 3)).astype(np.float32) + [0, 0, 0],
                     level=np.zeros(N, np.uint8), dL=np.zeros(N, np.float32),
                     feat=rng.normal(0, 0.3, size=(N, 32)).astype(np.float32),
                     offs=rng.normal(0, 0.5, size=(N, 10, 3)).astype(np.float32),
                     lv=rng.uniform(0.1, 0.3, size=(N, 3)).astype(np.float32), NL=1, k=10)
    return sc


def test_decode_bwd_matches_fd():
    sc = _tiny_scene()
    mlp = synth.decoder_mlp(seed=1, dist_scale=0.1)
    cam = synth.look_at_camera(np.array([0.0, -6.0, 1.5]), np.zeros(3), 32, 32, d_max=20.0)
    N = sc.N
    sel_idx = np.arange(N)[::2]
    sel_w = np.linspace(0.3, 1.0, len(sel_idx))
    # float64 copies that the FD perturbs
    scd = synth.Scene(pos=sc.pos.astype(np.float64), level=sc.level, dL=sc.dL,
                      feat=sc.feat.astype(np.float64), offs=sc.offs.astype(np.float64),
                      lv=sc.lv.astype(np.float64), NL=1, k=10)
    mlpd = synth.DecoderMLP(*[a.astype(np.float64) for a in mlp.arrays()])
    G = len(sel_idx) * 10
    rng = np.random.default_rng(4)
    wts = dict(dmeans=rng.normal(size=(G, 3)), dscales=rng.normal(size=(G, 3)),
               dquats=rng.normal(size=(G, 4)), dopac=rng.normal(size=G),
               dcolors=rng.normal(size=(G, 3)))
    base = oracle.decode(sel_idx, sel_w, scd, mlpd, cam)
    assert base["op_margin"].min() > 1e-4 or np.all(base["opac"] != 0)

    def f():
        o = oracle.decode(sel_idx, sel_w, scd, mlpd, cam)
        valid = o["opac"] > 0
        return float((o["means"] * wts["dmeans"]).sum() + (o["scales"] * wts["dscales"]).sum()
                     + (o["quats"] * wts["dquats"]).sum()
                     + (np.where(valid, o["opac"], 0) * wts["dopac"]).sum()
                     + (o["colors"] * wts["dcolors"]).sum())

    db = oracle.decode_bwd(sel_idx, sel_w, scd, mlpd, cam, wts)
    checks = [(scd.feat, db["dfeat"], [(0, 0), (0, 5), (2, 31), (4, 17)]),
              (scd.offs, db["doffs"], [(0, 0, 0), (2, 9, 2), (4, 3, 1)]),
              (scd.lv, db["dlv"], [(0, 0), (2, 1), (4, 2)]),
              (mlpd.w1, db["dw1"], [(0, 0, 0), (1, 5, 33), (2, 31, 35), (2, 3, 4)]),
              (mlpd.b1, db["db1"], [(0, 1), (1, 7), (2, 30)]),
              (mlpd.w2_op, db["dw2_op"], [(0, 0), (9, 31)]),
              (mlpd.b2_op, db["db2_op"], [(3,)]),
              (mlpd.w2_col, db["dw2_col"], [(0, 0), (29, 31)]),
              (mlpd.b2_col, db["db2_col"], [(17,)]),
              (mlpd.w2_cov, db["dw2_cov"], [(0, 0), (3, 2), (69, 31), (36, 11)]),
              (mlpd.b2_cov, db["db2_cov"], [(5,), (66,)])]
    for arr, grad, idxs in checks:
        for ix in idxs:
            assert grad[ix] == pytest.approx(_fd(f, arr, ix), rel=1e-5, abs=1e-7), (ix,)
    # unselected anchors get nothing
    assert np.all(db["dfeat"][1::2] == 0)


def test_full_render_grad_matches_fd():
    """Finite differences through select -> decode -> project -> lists -> blend."""
    rng = np.random.default_rng(11)
    N = 24
    pos = np.concatenate([rng.uniform(-1.5, 1.5, size=(N, 2)), rng.uniform(-0.3, 0.3, (N, 1))], 1)
    sc = synth.Scene(pos=pos, level=np.zeros(N, np.uint8), dL=np.zeros(N),
                     feat=rng.normal(0, 0.3, size=(N, 32)), offs=rng.normal(0, 0.5, (N, 10, 3)),
                     lv=rng.uniform(0.08, 0.15, size=(N, 3)), NL=2, k=10)
    mlp = synth.decoder_mlp(seed=5, dist_scale=0.1)
    mlpd = synth.DecoderMLP(*[a.astype(np.float64) for a in mlp.arrays()])
    cam = synth.look_at_camera(np.array([0.0, -5.0, 2.0]), np.zeros(3), 32, 32, d_max=8.0)
    bg = np.array([0.2, 0.1, 0.3])
    fr = oracle.render(sc, mlpd, cam, infer=True, bg=bg)
    assert len(fr.sel_idx) == N and fr.out["px_margin"].min() > 1e-5
    dimg = np.random.default_rng(12).normal(size=(3, 32, 32))

    def f():
        r = oracle.render(sc, mlpd, cam, infer=True, bg=bg)
        return float((r.out["img"] * dimg).sum())

    gr = oracle.render_grad(sc, mlpd, cam, fr, dimg, bg=bg)
    checks = [(sc.feat, gr["dfeat"], [(0, 0), (3, 12), (10, 31)]),
              (sc.offs, gr["doffs"], [(1, 0, 0), (5, 7, 2)]),
              (sc.lv, gr["dlv"], [(2, 0), (7, 2)]),
              (mlpd.w1, gr["dw1"], [(0, 3, 4), (1, 10, 33), (2, 0, 35)]),
              (mlpd.w2_cov, gr["dw2_cov"], [(1, 1), (45, 20)]),
              (mlpd.b2_op, gr["db2_op"], [(2,)]),
              (mlpd.w2_col, gr["dw2_col"], [(4, 9)])]
    for arr, grad, idxs in checks:
        for ix in idxs:
            assert grad[ix] == pytest.approx(_fd(f, arr, ix), rel=2e-5, abs=1e-6), (ix,)
