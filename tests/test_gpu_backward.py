"""GPU parity of the training path: blend/project/decode backward, L1 loss and Adam against
the FP64 oracle, the whole-chain gradient of a training view, and a finite-difference check
through the GPU forward at the 500k-anchor street-grid scale."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import cuda, lib_ready, to_np_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    return lib_ready()


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _close_frac(got, ref, rel=1e-3, floor_frac=1e-3):
    """Fraction of entries within rel of the reference, with an absolute floor of
    floor_frac x the reference's RMS (gradients near zero)."""
    got, ref = np.asarray(got, np.float64).ravel(), np.asarray(ref, np.float64).ravel()
    floor = floor_frac * np.sqrt(np.mean(ref ** 2)) + 1e-30
    return float(np.mean(np.abs(got - ref) <= rel * np.abs(ref) + floor))


def test_blend_bwd_matches_oracle(abi, torch):
    W, H, gx, gy = 72, 40, 5, 3
    r = synth.random_records(3, 300, W, H, sigma=(0.8, 10.0), opac=(0.05, 0.95))
    G = 300
    order = np.argsort(r["depth"], kind="stable")
    T = gx * gy
    lst = np.tile(order, T).astype(np.int64)
    start = np.arange(T + 1, dtype=np.int64) * G
    uv = np.stack([r["u"], r["v"]], 1)
    bg = (0.05, 0.1, 0.2)
    dimg = np.random.default_rng(5).normal(size=(3, H, W)).astype(np.float32)
    ref = oracle.blend_bwd(W, H, start, lst, uv, r["conic"], r["opac"], r["colors"], bg, dimg)
    rec = np.zeros((G, 12), np.float32)
    rec[:, 0], rec[:, 1] = r["u"], r["v"]
    rec[:, 2:4] = r["conic"][:, 0:2]
    rec[:, 4], rec[:, 5] = r["conic"][:, 2], r["opac"]
    rec[:, 6:9] = r["colors"]
    rec[:, 11] = -np.log(255.0 * r["opac"].astype(np.float64))
    tr = cuda(np.stack([start[:-1], start[1:]], 1).astype(np.int32))
    img = torch.zeros(3, H, W, device="cuda")
    Tf = torch.zeros(H, W, device="cuda")
    nl = torch.zeros(H, W, dtype=torch.int32, device="cuda")
    rec_t, lst_t = cuda(rec), cuda(lst.astype(np.int32))
    abi.blend_fwd(rec_t, lst_t, tr, W, H, bg, img, Tf, nl)
    drec = torch.zeros(G, 9, device="cuda")
    abi.blend_bwd(rec_t, lst_t, tr, W, H, bg, Tf, nl, cuda(dimg), drec)
    torch.cuda.synchronize()
    d = drec.cpu().numpy()
    assert _close_frac(d[:, 0:2], ref["duv"]) > 0.99
    assert _close_frac(d[:, 2:5], ref["dconic"]) > 0.99
    assert _close_frac(d[:, 5], ref["dopac"]) > 0.99
    assert _close_frac(d[:, 6:9], ref["dcolors"]) > 0.99
    # aggregate agreement over everything
    for a, b in ((d[:, 0:2], ref["duv"]), (d[:, 5], ref["dopac"]), (d[:, 6:9], ref["dcolors"])):
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b)


def test_project_bwd_matches_oracle(abi, torch):
    W, H = 160, 120
    cam = synth.look_at_camera(np.array([1.0, -8.0, 3.0]), np.zeros(3), W, H, d_max=30.0)
    g = synth.random_gaussians(7, 5000, cam, depth=(1.0, 30.0), scale=(0.02, 1.0))
    ref_p = oracle.project(g["means"], g["scales"], g["quats"], g["opac"], cam)
    G = 5000
    gt = {k: cuda(v) for k, v in g.items()}
    rec = torch.zeros(G, 12, device="cuda")
    dk = torch.zeros(G, dtype=torch.int32, device="cuda")
    rect = torch.zeros(G, 2, dtype=torch.int32, device="cuda")
    tiles = torch.zeros(G, dtype=torch.int32, device="cuda")
    abi.project_bin(gt, G, 0, cam, rec, dk, rect, tiles)
    rng = np.random.default_rng(8)
    drec = rng.normal(size=(G, 9)).astype(np.float32)
    drec[:, 2:5] *= 20.0
    dm = torch.zeros(G, 3, device="cuda")
    ds = torch.zeros(G, 3, device="cuda")
    dq = torch.zeros(G, 4, device="cuda")
    abi.project_bwd(gt, G, 0, cam, rect, cuda(drec), dm, ds, dq)
    torch.cuda.synchronize()
    vis = (ref_p["rect"][:, 2] > ref_p["rect"][:, 0]) & (ref_p["mpx"] > 1e-3)
    ref = oracle.project_bwd(g["means"], g["scales"], g["quats"], ref_p["rect"], cam,
                             drec[:, 0:2], drec[:, 2:5])
    for got, want in ((dm, ref["dmeans"]), (ds, ref["dscales"]), (dq, ref["dquats"])):
        a = got.cpu().numpy()[vis]
        b = want[vis]
        assert _close_frac(a, b, rel=2e-3) > 0.995
        assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(b)
    culled = (ref_p["rect"][:, 2] <= ref_p["rect"][:, 0]) & (ref_p["mpx"] > 1e-3)
    assert np.all(dm.cpu().numpy()[culled] == 0)


def _mlp_tensors(mlp):
    names = ("w1", "b1", "w2_op", "b2_op", "w2_col", "b2_col", "w2_cov", "b2_cov")
    return {n: cuda(a) for n, a in zip(names, mlp.arrays())}, names


def _bf16(x):
    """Round to bfloat16 (nearest, ties to even), returned as float64."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _bf16_decode_grads(sel, w, sc, mlp, cam, grads):
    """Feature and first-layer gradients of the decoders with the operands of the four
    tensor-core products rounded to BF16 and everything else exact: the arithmetic the BF16
    backward performs.  Their distance to the FP64 oracle is the error BF16 rounding alone
    causes on these inputs."""
    W1, b1, W2op, b2op, W2col, b2col, W2cov, b2cov = [np.asarray(a, np.float64)
                                                       for a in mlp.arrays()]
    W1, b1 = W1.reshape(96, 36), b1.reshape(96)
    W2 = np.zeros((110, 96))
    W2[0:10, 0:32], W2[10:40, 32:64], W2[40:110, 64:96] = W2op, W2col, W2cov
    b2 = np.concatenate([b2op, b2col, b2cov])
    M = len(sel)
    dv = sc.pos[sel].astype(np.float64) - cam.campos.astype(np.float64)
    d = np.linalg.norm(dv, axis=1)
    Z = np.concatenate([sc.feat[sel].astype(np.float64), dv / d[:, None], d[:, None]], 1)
    lvv = sc.lv[sel].astype(np.float64)
    hp = _bf16(Z) @ _bf16(W1).T + b1
    y = _bf16(np.maximum(hp, 0)) @ _bf16(W2).T + b2
    g = lambda k: grads[k].astype(np.float64).reshape(M, 10, -1)
    dy = np.zeros_like(y)
    th = np.tanh(y[:, 0:10])
    wv = w.astype(np.float64)[:, None]
    dy[:, 0:10] = np.where(wv * th > 0, g("dopac")[..., 0] * wv * (1 - th ** 2), 0)
    sg = 1 / (1 + np.exp(-y[:, 10:40]))
    dy[:, 10:40] = g("dcolors").reshape(M, 30) * sg * (1 - sg)
    cov = y[:, 40:110].reshape(M, 10, 7)
    s3 = 1 / (1 + np.exp(-cov[..., :3]))
    dcov = np.zeros_like(cov)
    dcov[..., :3] = g("dscales") * lvv[:, None, :] * s3 * (1 - s3)
    q = cov[..., 3:]
    n = np.linalg.norm(q, axis=-1, keepdims=True)
    qn = q / n
    gq = g("dquats")
    dcov[..., 3:] = (gq - qn * (qn * gq).sum(-1, keepdims=True)) / n
    dy[:, 40:110] = dcov.reshape(M, 70)
    dp = np.where(hp > 0, _bf16(dy) @ _bf16(W2), 0)
    dz = _bf16(dp) @ _bf16(W1)[:, :32]
    dfeat = np.zeros((sc.N, 32))
    np.add.at(dfeat, sel, dz)
    return {"dfeat": dfeat, "dw1": (dp.T @ Z).reshape(3, 32, 36), "db1": dp.sum(0).reshape(3, 32)}


def _big_scene(N, seed):
    rng = np.random.default_rng(seed)
    return synth.Scene(pos=rng.uniform(-30, 30, size=(N, 3)).astype(np.float32),
                       level=rng.integers(0, 4, N).astype(np.uint8),
                       dL=np.zeros(N, np.float32),
                       feat=rng.normal(0, 0.1, size=(N, 32)).astype(np.float32),
                       offs=rng.normal(0, 0.5, size=(N, 10, 3)).astype(np.float32),
                       lv=rng.uniform(0.1, 1.0, size=(N, 3)).astype(np.float32), NL=4)


# 900 anchors: one partial block; 40,001: many blocks of the row pass and many chunks of the
# weight pass (split over anchors), with a ragged last chunk.  bf16: the tensor-core row pass
# (BF16 operands: inputs, weights, hidden activations and output gradients rounded to 2^-9
# relative; FP32 accumulation), compared with the FP64 oracle at 2e-2 relative.
@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("M", [900, 40_001])
def test_decode_bwd_matches_oracle(abi, torch, M, bf16):
    if M <= 4096:
        sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
        cam = cams[0]
    else:
        sc = _big_scene(M + 5000, 9)
        mlp = synth.decoder_mlp(seed=3, dist_scale=1.0 / 60.0)
        cam = synth.look_at_camera(np.array([40.0, -45.0, 20.0]), np.zeros(3), 128, 128,
                                   d_max=120.0)
    rng = np.random.default_rng(2)
    sel = np.sort(rng.choice(sc.N, size=M, replace=False)).astype(np.int64)
    w = rng.uniform(0.05, 1.0, size=M).astype(np.float32)
    G = M * 10
    grads = dict(dmeans=rng.normal(size=(G, 3)), dscales=rng.normal(size=(G, 3)),
                 dquats=rng.normal(size=(G, 4)), dopac=rng.normal(size=G),
                 dcolors=rng.normal(size=(G, 3)))
    grads = {k: v.astype(np.float32) for k, v in grads.items()}
    ref = oracle.decode_bwd(sel, w, sc, mlp, cam, grads)
    counts = np.zeros(8, np.uint32)
    counts[0], counts[1] = M, G
    drec = np.zeros((G, 9), np.float32)
    drec[:, 5] = grads["dopac"]
    drec[:, 6:9] = grads["dcolors"]
    mt, names = _mlp_tensors(mlp)
    dmlp = {n: torch.zeros_like(t) for n, t in mt.items()}
    dfeat = torch.zeros(sc.N, 32, device="cuda")
    doffs = torch.zeros(sc.N, 10, 3, device="cuda")
    dlv = torch.zeros(sc.N, 3, device="cuda")
    cap = M + 77                      # capacity above the device count
    scr = torch.empty(abi.decode_bwd_scratch_bytes(cap), dtype=torch.uint8, device="cuda")
    args = (cuda(sc.pos), cuda(sc.feat), cuda(sc.offs), cuda(sc.lv), sc.N, mt, cam,
            cuda(np.concatenate([sel, np.zeros(77, np.int64)]).astype(np.int32)),
            cuda(np.concatenate([w, np.zeros(77, np.float32)])), cap,
            cuda(counts.view(np.int32)), cuda(grads["dmeans"]), cuda(grads["dscales"]),
            cuda(grads["dquats"]), cuda(drec), dfeat, doffs, dlv, dmlp, scr)
    ct = args[10]
    abi.decode_bwd(*args, bf16=bf16)
    torch.cuda.synchronize()
    assert to_np_u32(ct)[6] == 0                   # no tensor-core wait expired
    # opacity-sign knife edges would drop a Gaussian's opacity gradient on one side only
    dec = oracle.decode(sel, w, sc, mlp, cam)
    keep_g = dec["op_margin"] > 1e-5
    assert keep_g.mean() > 0.999
    base_tol = 2e-2 if bf16 else 1e-4
    errs = {}
    emu_bound = {}
    if bf16:
        # dfeat, dw1 and db1 pass dy and dp through BF16 products; their bound is the error
        # that BF16 rounding alone gives on these inputs (cancellation in the random upstream
        # gradients makes it a few percent), plus FP32 accumulation slack
        emu = _bf16_decode_grads(sel, w, sc, mlp, cam, grads)
        got = {"dfeat": dfeat.cpu().numpy(), "dw1": dmlp["w1"].cpu().numpy(),
               "db1": dmlp["b1"].cpu().numpy()}
        for name in emu:
            b = ref[name]
            emu_err = np.linalg.norm(emu[name] - b) / np.linalg.norm(b)
            emu_bound[name] = 1.1 * emu_err + 1e-3
            err = np.linalg.norm(got[name] - b) / np.linalg.norm(b)
            assert err <= emu_bound[name], (name, err, emu_err)
            assert np.linalg.norm(got[name] - emu[name]) <= 2e-2 * np.linalg.norm(b), name
            print(f"decode_bwd bf16 M={M}: {name} error {err:.4f}, BF16 emulation {emu_err:.4f}")
    if keep_g.all() or bf16:
        for name, got in (("dfeat", dfeat), ("doffs", doffs), ("dlv", dlv)):
            if name in emu_bound:
                continue
            a, b = got.cpu().numpy(), ref[name]
            errs[name] = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert errs[name] <= base_tol, name
    for n in names:
        a, b = dmlp[n].cpu().numpy(), ref["d" + n]
        tol = emu_bound.get("d" + n, base_tol if keep_g.all() else max(base_tol, 1e-3))
        errs[n] = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert errs[n] <= tol, n
    if bf16:
        print(f"decode_bwd bf16 M={M} relative errors:",
              {k: f"{v:.1e}" for k, v in errs.items()})
    # a second call accumulates
    abi.decode_bwd(*args, bf16=bf16)
    torch.cuda.synchronize()
    a, b = dmlp["w1"].cpu().numpy(), 2 * ref["dw1"]
    tol1 = emu_bound.get("dw1", base_tol if keep_g.all() else max(base_tol, 1e-3))
    assert np.linalg.norm(a - b) <= 2 * tol1 * np.linalg.norm(b)


def test_loss_and_adam_match_oracle(abi, torch):
    rng = np.random.default_rng(3)
    img = rng.uniform(size=(3, 40, 50)).astype(np.float32)
    tgt = rng.uniform(size=(3, 40, 50)).astype(np.float32)
    dimg = torch.zeros(3, 40, 50, device="cuda")
    loss = torch.zeros(1, device="cuda")
    abi.loss_l1(cuda(img), cuda(tgt), img.size, dimg, loss)
    torch.cuda.synchronize()
    L, g = oracle.l1_loss(img, tgt)
    assert abs(loss.item() - L) <= 1e-6
    np.testing.assert_allclose(dimg.cpu().numpy(), g, rtol=1e-6)
    p = rng.normal(size=1000).astype(np.float32)
    m = np.zeros(1000, np.float32)
    v = np.zeros(1000, np.float32)
    pt, mt_, vt = cuda(p), cuda(m), cuda(v)
    po, mo, vo = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for step in range(1, 6):
        gr = rng.normal(size=1000).astype(np.float32)
        gt = cuda(gr)
        abi.adam(pt, gt, mt_, vt, 1000, 1e-2, 0.9, 0.999, 1e-8, step, True)
        po, mo, vo = oracle.adam(po, gr, mo, vo, 1e-2, 0.9, 0.999, 1e-8, step)
        torch.cuda.synchronize()
        assert np.all(gt.cpu().numpy() == 0)
    np.testing.assert_allclose(pt.cpu().numpy(), po, rtol=1e-5, atol=1e-6)


def test_training_view_gradient_matches_oracle(abi, torch):
    """Whole chain for one training view of the 4k-anchor cube (L1 against a seeded target)."""
    from paper_2403_17898_gb300.render import Trainer
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    cam = cams[0]
    target = np.random.default_rng(1).uniform(size=(3, 128, 128)).astype(np.float32)
    tr = Trainer(sc, mlp, 128, 128)
    c = tr.render(cam, infer=False)
    assert c.overflow == 0
    tr.zero_grad()
    tr.backward_view(cam, cuda(target))
    torch.cuda.synchronize()
    fr = oracle.render(sc, mlp, cam, infer=False)
    L, dimg = oracle.l1_loss(fr.out["img"], target)
    assert abs(tr.loss.item() - L) <= 1e-5
    ref = oracle.render_grad(sc, mlp, cam, fr, dimg)
    pairs = [("dfeat", tr.grads["feat"]), ("doffs", tr.grads["offs"]), ("dlv", tr.grads["lv"])]
    pairs += [("d" + n, tr.dmlp[n]) for n in tr.mlp]
    for name, got in pairs:
        a, b = got.cpu().numpy(), ref[name]
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err <= 5e-3, (name, err)
    # per-anchor feature gradients agree almost everywhere
    assert _close_frac(tr.grads["feat"].cpu().numpy(), ref["dfeat"], rel=1e-2) > 0.98


def test_finite_difference_through_gpu_street_scale(abi, torch):
    """FD check of decoder-weight gradients through the FP32 GPU forward at the 500k-anchor,
    1600x900 street-grid scale.  The target is black, so L1 is the mean intensity: no pixel
    sits on the |.| kink and the FD quotient is not a cancelling sum of signs; the loss for
    the FD is summed in float64 on the host to keep accumulation noise below the signal.

    Only colour-decoder parameters are perturbed: they never move alpha.  Opacity and
    geometry parameters push (pixel, Gaussian) pairs across the alpha >= 1/255 skip and the
    T < 1e-4 stop; at this scale the resulting jumps (which the analytic gradient omits by
    definition) move a finite difference by several percent.  Those chains are checked
    against the oracle's analytic gradient instead (and the oracle against FD on scenes with
    no decision near a threshold)."""
    from paper_2403_17898_gb300.render import Trainer
    sc, mlp, cams = synth.CONFIGS["street500k_1600x900"]()
    cam = cams[10]
    target = torch.zeros(3, cam.H, cam.W, device="cuda")
    tr = Trainer(sc, mlp, cam.W, cam.H, sel_cap=200_000, pair_cap=4_000_000)
    c = tr.render(cam, infer=False)
    assert c.overflow == 0 and c.n_selected > 1000
    tr.zero_grad()
    tr.loss.zero_()
    tr.backward_view(cam, target)
    torch.cuda.synchronize()

    def loss_at():
        tr.enqueue(cam, infer=False)
        torch.cuda.synchronize()
        return float(tr.img.double().mean().item())

    assert abs(loss_at() - tr.loss.item()) <= 1e-5 * abs(loss_at())
    checks = [("b2_col", (4,)), ("b2_col", (17,)), ("b1", (1, 5)), ("b1", (1, 9)),
              ("w2_col", (5, 7)), ("w2_col", (22, 30)), ("w1", (1, 3, 4)), ("w1", (1, 10, 33))]
    for name, ix in checks:
        p = tr.mlp[name]
        g = float(tr.dmlp[name][ix].item())
        x0 = float(p[ix].item())
        # first-layer parameters move ReLU kinks: a smaller step keeps the quotient local
        h = 2e-3 if name in ("b1", "w1") else 0.02
        p[ix] = x0 + h
        lp = loss_at()
        p[ix] = x0 - h
        lm = loss_at()
        p[ix] = x0
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g) <= 0.03 * abs(g) + 1e-6, (name, ix, g, fd)


def test_adam_rows_match_oracle(abi, torch):
    """Adam over stamped rows against the oracle's row Adam over four steps with different
    touched sets (rows of 30 values, like the offsets): touched rows within FP32 rounding,
    untouched rows bit for bit unchanged, gradients of touched rows cleared."""
    rng = np.random.default_rng(11)
    N, L = 5000, 30
    p = rng.normal(size=(N, L)).astype(np.float32)
    pt, mt_, vt = cuda(p), torch.zeros(N, L, device="cuda"), torch.zeros(N, L, device="cuda")
    stamp = torch.zeros(N, dtype=torch.int32, device="cuda")
    po, mo, vo = p.astype(np.float64), np.zeros((N, L)), np.zeros((N, L))
    for step in range(1, 5):
        rows = np.sort(rng.choice(N, size=rng.integers(1, N // 3), replace=False))
        sel = cuda(rows.astype(np.int32))
        counts = np.zeros(8, np.uint32)
        counts[0] = len(rows)
        abi.stamp_selected(sel, cuda(counts.view(np.int32)), stamp, step)
        gr = np.zeros((N, L), np.float32)
        gr[rows] = rng.normal(size=(len(rows), L)).astype(np.float32)
        gt = cuda(gr)
        before = pt.cpu().numpy()
        abi.adam_rows(pt, gt, mt_, vt, stamp, step, 1e-2, 0.9, 0.999, 1e-8, step)
        po, mo, vo = oracle.adam_rows(po, gr, mo, vo, rows, 1e-2, 0.9, 0.999, 1e-8, step)
        torch.cuda.synchronize()
        got = pt.cpu().numpy()
        untouched = np.setdiff1d(np.arange(N), rows)
        assert np.array_equal(got[untouched], before[untouched])
        assert np.all(gt.cpu().numpy()[rows] == 0)
        np.testing.assert_allclose(got, po, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(mt_.cpu().numpy(), mo, rtol=1e-5, atol=1e-7)


def test_trainer_sparse_adam_touches_selected_rows_only(abi, torch):
    """One training step of the cube: anchors no view selected keep their features, offsets,
    l_v and Adam moments bit for bit; the selected ones move (a dense step would move every
    row with a nonzero first moment, here none yet)."""
    from paper_2403_17898_gb300.render import Trainer
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    cam = cams[0]
    target = cuda(np.random.default_rng(1).uniform(size=(3, 128, 128)).astype(np.float32))
    tr = Trainer(sc, mlp, 128, 128)
    assert tr.sparse_adam
    f0 = tr.feat.clone()
    tr.train_step([cam], [target])
    c = tr.counts()
    torch.cuda.synchronize()
    sel = to_np_u32(tr.sel_idx)[:c.n_selected].astype(np.int64)
    touched = np.zeros(sc.N, bool)
    touched[sel] = True
    moved = (tr.feat != f0).any(dim=1).cpu().numpy()
    assert moved.any() and not moved[~touched].any()
    assert np.array_equal(to_np_u32(tr.stamp)[touched], np.ones(touched.sum(), np.uint32))
    assert not tr.adam_m["feat"].cpu().numpy()[~touched].any()


def test_scan_nonfinite(abi, torch):
    """The opt-in non-finite scan: a clean buffer leaves the flag alone; a NaN or an infinity
    anywhere (ragged length, last element included) sets the requested bit."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=1_000_003).astype(np.float32)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    abi.scan_nonfinite(cuda(x), flag, 4)
    torch.cuda.synchronize()
    assert flag.item() == 0
    for pos, val in ((0, np.nan), (517_311, np.inf), (1_000_002, -np.inf)):
        y = x.copy()
        y[pos] = val
        flag.zero_()
        abi.scan_nonfinite(cuda(y), flag, 4)
        torch.cuda.synchronize()
        assert flag.item() == 4


@pytest.mark.parametrize("precision,tol", [("fp32", 5e-3), ("bf16", 6e-2)])
def test_training_view_gradient_street_scale(abi, torch, precision, tol):
    """One training view of the 500k-anchor street workload (1600x900, pose 10 of the
    zoom-out), L1 against a seeded target, through the forward and backward the benchmark
    times: features, offsets and l_v on a seeded sample of kept anchors and every decoder
    weight against the FP64 oracle's analytic gradient, relative L2 within the chain
    tolerance (FP32) or the BF16 bound (the decoder backward's BF16 products: ~3% on the
    feature and first-layer gradients, see the tensor-core decoder tests)."""
    from paper_2403_17898_gb300.render import Trainer
    sc, mlp, cams = synth.CONFIGS["street500k_1600x900"]()
    cam = cams[10]
    target = np.random.default_rng(1).uniform(size=(3, cam.H, cam.W)).astype(np.float32)
    tr = Trainer(sc, mlp, cam.W, cam.H, sel_cap=200_000, pair_cap=4_000_000,
                 precision=precision)
    c = tr.render(cam, infer=False)
    assert c.overflow == 0 and c.timeout == 0
    tr.zero_grad()
    tr.loss.zero_()
    tr.backward_view(cam, cuda(target))
    torch.cuda.synchronize()
    fr = oracle.render(sc, mlp, cam, infer=False)
    L, dimg = oracle.l1_loss(fr.out["img"], target)
    ref = oracle.render_grad(sc, mlp, cam, fr, dimg)
    kept = fr.sel_idx
    rng = np.random.default_rng(3)
    sample = np.sort(rng.choice(kept, size=min(4000, len(kept)), replace=False))
    assert len(kept) > 2000 and len(sample) >= 2000
    errs = {}
    for name, got in (("dfeat", tr.grads["feat"]), ("doffs", tr.grads["offs"]),
                      ("dlv", tr.grads["lv"])):
        a = got.cpu().numpy()[sample].astype(np.float64)
        b = ref[name][sample]
        errs[name] = np.linalg.norm(a - b) / np.linalg.norm(b)
    for n in tr.mlp:
        a, b = tr.dmlp[n].cpu().numpy().astype(np.float64), ref["d" + n]
        errs["d" + n] = np.linalg.norm(a - b) / np.linalg.norm(b)
    print(f"street500k view ({precision}): {c.n_selected} anchors, {c.n_pairs} pairs, loss "
          f"{tr.loss.item():.6f} vs {L:.6f}; gradient relative L2:",
          {k: f"{v:.2e}" for k, v in errs.items()})
    assert abs(tr.loss.item() - L) <= 1e-4 * L
    for k, v in errs.items():
        assert v <= tol, (k, v)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_pipelined_step_equals_sequential(abi, torch, precision):
    """The pipelined training step (two sets of per-view buffers; each view's backward on a
    second stream overlapping the next view's forward) accumulates the same gradients and
    loss as the sequential step, on 6 views of the 500k-anchor street at 1600x900 with
    L1 + D-SSIM (float atomics in the blend backward sum in varying order, hence the
    tolerance); its Adam update then runs without overflow or expired waits."""
    from paper_2403_17898_gb300.render import Trainer
    sc, mlp, cams = synth.CONFIGS["street500k_1600x900"]()
    views = cams[::5][:6]
    W, H = views[0].W, views[0].H
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4)
    tgts = [torch.rand(3, H, W, generator=gen, device="cuda") for _ in views]
    out = {}
    for pipe in (False, True):
        tr = Trainer(sc, mlp, W, H, ssim_lambda=0.2, sel_cap=60_000, pair_cap=2_000_000,
                     precision=precision)
        tr.pipeline = pipe
        for cam in views:
            assert tr.render(cam, infer=False).overflow == 0
        tr.zero_grad()
        tr.train_step(views, tgts, update=False)
        torch.cuda.synchronize()
        c = tr.counts()
        assert c.overflow == 0 and c.timeout == 0
        grads = {n: t.clone() for n, t in tr.grads.items()}
        grads.update({"mlp." + n: t.clone() for n, t in tr.dmlp.items()})
        out[pipe] = (grads, tr.loss.item())
        if pipe:
            tr.train_step(views, tgts)             # with the update
            torch.cuda.synchronize()
            c = tr.counts()
            assert c.overflow == 0 and c.timeout == 0
            assert all(torch.isfinite(t).all() for t in tr._anchor_params().values())
        del tr
    (g0, l0), (g1, l1) = out[False], out[True]
    assert abs(l0 - l1) <= 1e-5 * abs(l0)
    for n in g0:
        ref = torch.linalg.norm(g0[n])
        assert ref > 0, n
        assert torch.linalg.norm(g1[n] - g0[n]) <= 1e-4 * ref, n


def test_training_fits_rendered_targets(abi, torch):
    """Ten pipelined steps (4 views of the 500k-anchor street at 1600x900, L1 + D-SSIM, dense
    Adam at lr 1e-3) from a perturbed scene towards the views it rendered before the
    perturbation: the scene keeps drawing (pair counts within 10 % of the unperturbed ones),
    and after Adam's first steps, which move every weight by about lr whatever its gradient
    and so overshoot from this near-optimal start (0.0054 -> 0.029 in one run), the loss falls
    to under half its peak (0.0093 after ten steps in that run).  A step that drove the
    decoded opacities below zero, as noise targets do, fails the first check."""
    from paper_2403_17898_gb300.render import Trainer
    sc, mlp, cams = synth.CONFIGS["street500k_1600x900"]()
    views = cams[::7][:4]
    W, H = views[0].W, views[0].H
    tr = Trainer(sc, mlp, W, H, ssim_lambda=0.2, sel_cap=60_000, pair_cap=2_000_000,
                 precision="bf16")
    tgts, pairs0 = [], []
    for cam in views:
        c = tr.render(cam, infer=False)
        assert c.overflow == 0 and c.timeout == 0
        tgts.append(tr.img.clone())
        pairs0.append(c.n_pairs)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    tr.feat.add_(0.05 * torch.randn(tr.feat.shape, generator=gen, device="cuda"))
    losses = []
    for _ in range(10):
        tr.train_step(views, tgts)
        losses.append(tr.loss.item())
    c = tr.counts()
    assert c.overflow == 0 and c.timeout == 0
    print("fit losses", [round(x, 5) for x in losses])
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.5 * max(losses), losses
    pairs = [tr.render(cam, infer=False).n_pairs for cam in views]
    assert sum(pairs) >= 0.9 * sum(pairs0), (pairs, pairs0)
