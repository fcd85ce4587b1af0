"""Appearance codes (Sec. 4.4: a learnable code per anchor that only the colour decoder sees)
through the CUDA path, against the FP64 oracle.

Forward: ogs_decode (FP32), ogs_decode_bf16 and the fused ogs_decode_project_bf16 with codes,
at the tolerances of the plain decoders' parity tests (the code adds 8 inputs of the same
scale to the colour decoder's first layer).  The code may change the colours only: opacity,
scales, rotations and positions are the same bits as without codes.  Zero codes give the
plain decoder's colours, and the fused kernel equals the two-call path bit for bit.
Backward: ogs_decode_bwd (FP32) and ogs_decode_bwd_bf16 (tensor cores) give the code
gradients (dapp) and the code weights' gradient (dw1_app) next to every other gradient.
Training: a whole training view through the Trainer, and pruning keeps codes aligned."""
import copy

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import cuda, lib_ready, to_np_u32

pytestmark = pytest.mark.gpu

NAMES = ("w1", "b1", "w2_op", "b2_op", "w2_col", "b2_col", "w2_cov", "b2_cov")
GAUSS = ("means", "scales", "quats", "opac", "colors")


@pytest.fixture(scope="module")
def abi():
    return lib_ready()


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _mlp(mlp, app):
    """Decoder struct with (or, app None, without) appearance codes."""
    from paper_2403_17898_gb300 import abi as A
    t = {n: cuda(a) for n, a in zip(NAMES, mlp.arrays())}
    if app is not None:
        t["w1_app"] = cuda(mlp.w1_app)
        keep = (t, cuda(app))
        return A.mlp_struct(t, app=keep[1]), keep
    return A.mlp_struct(t), (t,)


def _bufs(torch, G):
    return {"means": torch.zeros(G, 3, device="cuda"), "scales": torch.zeros(G, 3, device="cuda"),
            "quats": torch.zeros(G, 4, device="cuda"), "opac": torch.zeros(G, device="cuda"),
            "colors": torch.zeros(G, 3, device="cuda")}


def _decode(abi, torch, sc, mlp, cam, sel, w, kind, app):
    """kind: "fp32" (ogs_decode), "bf16" (ogs_decode_bf16) or "fused" (ogs_decode_project_bf16
    writing the Gaussians too).  Returns the Gaussians (and records for "fused")."""
    M = len(sel)
    G = max(M, 1) * 10
    counts = np.zeros(8, np.uint32)
    counts[0], counts[1] = M, M * 10
    ct = cuda(counts.view(np.int32))
    m, keep = _mlp(mlp, app)
    out = _bufs(torch, G)
    args = (cuda(sc.pos), cuda(sc.feat), cuda(sc.offs), cuda(sc.lv), sc.N, m, cam,
            cuda(np.resize(sel, max(M, 1)).astype(np.int32)),
            cuda(np.resize(np.asarray(w, np.float32), max(M, 1))), max(M, 1), ct)
    rec = None
    if kind == "fp32":
        abi.decode(*args, out)
    elif kind == "bf16":
        abi.decode_bf16(*args, out)
    else:
        gx, gy = (cam.W + 15) // 16, (cam.H + 15) // 16
        rec = torch.zeros(G, 12, device="cuda")
        dk = torch.zeros(G, dtype=torch.int32, device="cuda")
        rect = torch.zeros(G, 2, dtype=torch.int32, device="cuda")
        tiles = torch.zeros(G, dtype=torch.int32, device="cuda")
        tc = torch.zeros(gx * gy, dtype=torch.int32, device="cuda")
        scr = torch.empty(abi.decode_project_scratch_bytes(), dtype=torch.uint8, device="cuda")
        abi.decode_project_bf16(*args, rec, dk, rect, tiles, scr, out=out, tile_count=tc)
    torch.cuda.synchronize()
    assert to_np_u32(ct)[6] == 0                       # no bounded wait expired
    got = {k: v.cpu().numpy()[:M * 10] for k, v in out.items()}
    if rec is not None:
        got["rec"] = rec.cpu().numpy()[:M * 10]
    return got


def _pick(sc, M, seed):
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(sc.N, size=M, replace=False)).astype(np.int64)
    return sel, rng.uniform(0.05, 1.0, size=M)


@pytest.mark.parametrize("kind", ["fp32", "bf16", "fused"])
@pytest.mark.parametrize("M", [1, 127, 777, 3000])
def test_decode_with_codes_matches_oracle(abi, torch, kind, M):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    sa, ma = synth.with_appearance(sc, mlp, seed=M)
    cam = cams[0]
    sel, w = _pick(sc, M, 40 + M)
    ref = oracle.decode(sel, w, sa, ma, cam)
    plain = oracle.decode(sel, w, sc, mlp, cam)
    got = _decode(abi, torch, sa, ma, cam, sel, w, kind, sa.app)
    col = np.abs(got["colors"].astype(np.float64) - ref["colors"]).max()
    shift = np.abs(ref["colors"] - plain["colors"]).max()
    print(f"{kind} M={M}: colour error {col:.2e}, code's colour shift {shift:.2e}")
    tol = 2e-5 if kind == "fp32" else 1e-2
    assert col <= tol
    if M >= 127:
        assert shift > 50 * col                       # the code moves colours far beyond the error
    # everything but the colours is the plain decoder's, bit for bit
    base = _decode(abi, torch, sc, mlp, cam, sel, w, kind, None)
    for k in ("means", "scales", "quats", "opac"):
        assert np.array_equal(got[k], base[k]), k
    if kind == "fused":
        # records of the fused call equal its own Gaussians' projection (same colours)
        vis = got["rec"][:, 5] > 0
        assert np.array_equal(got["rec"][vis, 6:8], got["colors"][vis, 0:2])
        assert np.array_equal(got["rec"][vis, 8], got["colors"][vis, 2])


@pytest.mark.parametrize("kind", ["fp32", "bf16", "fused"])
def test_zero_codes_give_plain_colours(abi, torch, kind):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    sa, ma = synth.with_appearance(sc, mlp, seed=5)
    sel, w = _pick(sc, 777, 5)
    zero = np.zeros_like(sa.app)
    got = _decode(abi, torch, sa, ma, cams[0], sel, w, kind, zero)
    base = _decode(abi, torch, sc, mlp, cams[0], sel, w, kind, None)
    for k in GAUSS:
        assert np.array_equal(got[k], base[k]), k


def test_fused_with_codes_equals_two_calls_city(abi, torch):
    """The fused call against ogs_decode_bf16 (both with codes) on ~100k city anchors."""
    sc, mlp, cams = synth.CONFIGS["city2M_1080p"]()
    sa, ma = synth.with_appearance(sc, mlp, seed=3)
    cam = cams[40]
    sel, w, _ = oracle.lod_select(sc.pos, sc.level, sc.dL, sc.NL, cam, True)
    a = _decode(abi, torch, sa, ma, cam, sel, w, "bf16", sa.app)
    b = _decode(abi, torch, sa, ma, cam, sel, w, "fused", sa.app)
    for k in GAUSS:
        assert np.array_equal(a[k], b[k]), k
    # sampled anchors against the oracle
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(len(sel), size=500, replace=False))
    ref = oracle.decode(sel[pick], w[pick], sa, ma, cam)
    rows = (pick[:, None] * 10 + np.arange(10)).ravel()
    assert np.abs(b["colors"][rows] - ref["colors"]).max() <= 1e-2


@pytest.mark.parametrize("M", [900, 40_001])
def test_decode_bwd_with_codes_matches_oracle(abi, torch, M):
    if M <= 4096:
        sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
        cam = cams[0]
    else:
        rng0 = np.random.default_rng(9)
        N = M + 5000
        sc = synth.Scene(pos=rng0.uniform(-30, 30, size=(N, 3)).astype(np.float32),
                         level=rng0.integers(0, 4, N).astype(np.uint8),
                         dL=np.zeros(N, np.float32),
                         feat=rng0.normal(0, 0.1, size=(N, 32)).astype(np.float32),
                         offs=rng0.normal(0, 0.5, size=(N, 10, 3)).astype(np.float32),
                         lv=rng0.uniform(0.1, 1.0, size=(N, 3)).astype(np.float32), NL=4)
        mlp = synth.decoder_mlp(seed=3, dist_scale=1.0 / 60.0)
        cam = synth.look_at_camera(np.array([40.0, -45.0, 20.0]), np.zeros(3), 128, 128,
                                   d_max=120.0)
    sa, ma = synth.with_appearance(sc, mlp, seed=M)
    rng = np.random.default_rng(2)
    sel = np.sort(rng.choice(sc.N, size=M, replace=False)).astype(np.int64)
    w = rng.uniform(0.05, 1.0, size=M).astype(np.float32)
    G = M * 10
    grads = dict(dmeans=rng.normal(size=(G, 3)), dscales=rng.normal(size=(G, 3)),
                 dquats=rng.normal(size=(G, 4)), dopac=rng.normal(size=G),
                 dcolors=rng.normal(size=(G, 3)))
    grads = {k: v.astype(np.float32) for k, v in grads.items()}
    ref = oracle.decode_bwd(sel, w, sa, ma, cam, grads)
    dec = oracle.decode(sel, w, sa, ma, cam)
    keep_g = dec["op_margin"] > 1e-5
    from paper_2403_17898_gb300 import abi as A
    counts = np.zeros(8, np.uint32)
    counts[0], counts[1] = M, G
    drec = np.zeros((G, 9), np.float32)
    drec[:, 5] = grads["dopac"]
    drec[:, 6:9] = grads["dcolors"]
    m, keep = _mlp(ma, sa.app)
    dt = {n: torch.zeros_like(t) for n, t in keep[0].items()}
    dapp = torch.zeros(sc.N, sa.app.shape[1], device="cuda")
    dm = A.mlp_struct(dt, app=dapp)
    dfeat = torch.zeros(sc.N, 32, device="cuda")
    doffs = torch.zeros(sc.N, 10, 3, device="cuda")
    dlv = torch.zeros(sc.N, 3, device="cuda")
    scr = torch.empty(abi.decode_bwd_scratch_bytes(M), dtype=torch.uint8, device="cuda")
    args = (cuda(sa.pos), cuda(sa.feat), cuda(sa.offs), cuda(sa.lv), sc.N, m, cam,
            cuda(sel.astype(np.int32)), cuda(w), M, cuda(counts.view(np.int32)),
            cuda(grads["dmeans"]), cuda(grads["dscales"]), cuda(grads["dquats"]), cuda(drec),
            dfeat, doffs, dlv, dm, scr)
    abi.decode_bwd(*args)
    torch.cuda.synchronize()
    tol = 1e-4 if keep_g.all() else 1e-3
    errs = {}
    pairs = [("dapp", dapp), ("dw1_app", dt["w1_app"]), ("dfeat", dfeat), ("dlv", dlv)]
    pairs += [("d" + n, dt[n]) for n in NAMES]
    for name, got in pairs:
        a, b = got.cpu().numpy(), ref[name]
        errs[name] = np.linalg.norm(a - b) / np.linalg.norm(b)
    print(f"decode_bwd with codes M={M}:", {k: f"{v:.1e}" for k, v in errs.items()})
    for name, e in errs.items():
        assert e <= tol, (name, e)
    # only the selected anchors get a code gradient
    other = np.setdiff1d(np.arange(sc.N), sel)
    assert not dapp.cpu().numpy()[other].any()
    # the tensor-core backward: BF16 operands (the code and its weights included); its
    # feature-side gradients carry the BF16 rounding of dy and dp (a few percent on these
    # random upstream gradients, see test_gpu_backward), the weight gradients less
    for t in [dapp, dfeat, doffs, dlv] + list(dt.values()):
        t.zero_()
    abi.decode_bwd(*args, bf16=True)
    torch.cuda.synchronize()
    errs = {}
    for name, got in pairs:
        a, b = got.cpu().numpy(), ref[name]
        errs[name] = np.linalg.norm(a - b) / np.linalg.norm(b)
    print(f"decode_bwd bf16 with codes M={M}:", {k: f"{v:.1e}" for k, v in errs.items()})
    for name, e in errs.items():
        assert e <= 6e-2, (name, e)
    assert not dapp.cpu().numpy()[other].any()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_training_view_with_codes_matches_oracle(abi, torch, precision):
    """Whole chain for one training view of the 4k-anchor cube with codes (the BF16 form runs
    the tensor-core decoder backward)."""
    from paper_2403_17898_gb300.render import Trainer
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    sa, ma = synth.with_appearance(sc, mlp, seed=11)
    cam = cams[0]
    target = np.random.default_rng(1).uniform(size=(3, 128, 128)).astype(np.float32)
    tr = Trainer(sa, ma, 128, 128, precision=precision)
    c = tr.render(cam, infer=False)
    assert c.overflow == 0
    tr.zero_grad()
    tr.backward_view(cam, cuda(target))
    torch.cuda.synchronize()
    fr = oracle.render(sa, ma, cam, infer=False)
    ref = oracle.render_grad(sa, ma, cam, fr, oracle.l1_loss(fr.out["img"], target)[1])
    tol = 5e-3 if precision == "fp32" else 5e-2
    for name, got in (("dapp", tr.grads["app"]), ("dw1_app", tr.dmlp["w1_app"]),
                      ("dfeat", tr.grads["feat"])):
        a, b = got.cpu().numpy(), ref[name]
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        print(f"training view ({precision}) {name}: relative error {err:.2e}")
        assert err <= tol, (name, err)
    # an optimiser step moves the codes of the selected anchors only
    before = tr.app.clone()
    tr.optimizer_step()
    torch.cuda.synchronize()
    moved = (tr.app != before).any(dim=1).cpu().numpy()
    assert moved.any()
    assert not moved[np.abs(ref["dapp"]).sum(1) == 0].any()


def test_prune_keeps_codes_aligned(abi, torch):
    """Training with codes, then view-frequency pruning: the codes (and their Adam state) are
    compacted with the anchors, and the Trainer renders from the compacted codes: its frame
    equals a fresh renderer's built from the pruned arrays, bit for bit."""
    from paper_2403_17898_gb300.render import Renderer, Trainer
    sc, mlp, _ = synth.CONFIGS["cube4k_128"]()
    sa, ma = synth.with_appearance(sc, mlp, seed=12)
    rng = np.random.default_rng(3)
    views = [synth.look_at_camera(rng.uniform(-15, 15, 3) + np.array([0, 0, 12.0]),
                                  rng.uniform(-2, 2, 3), 128, 128, d_max=30.0) for _ in range(5)]
    tr = Trainer(sa, ma, 128, 128, track_view_frequency=True)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    tgts = [torch.rand(3, 128, 128, generator=gen, device="cuda") for _ in views]
    tr.train_step(views, tgts)
    count = tr.sel_count.cpu().numpy().astype(np.int64)
    keep_ref = oracle.prune_by_view_frequency(count, len(views), 0.4)
    app0 = tr.app.cpu().numpy()
    assert not np.array_equal(app0, sa.app)            # the step trained the codes
    m_app = tr.adam_m["app"].cpu().numpy()
    n = tr.prune(0.4)
    assert n == len(keep_ref) and 0 < n < sc.N
    assert np.array_equal(tr.app.cpu().numpy(), app0[keep_ref])
    assert np.array_equal(tr.adam_m["app"].cpu().numpy(), m_app[keep_ref])
    tr.train_step(views, tgts)                         # the pruned set still trains
    assert tr.counts().timeout == 0
    sp = copy.copy(sa)
    for name in ("pos", "level", "dL", "feat", "offs", "lv", "app"):
        setattr(sp, name, getattr(tr, name).cpu().numpy())
    mp = copy.copy(ma)
    for name in NAMES + ("w1_app",):
        setattr(mp, name, tr.mlp[name].cpu().numpy())
    fresh = Renderer(sp, mp, 128, 128)
    for v in views[:2]:
        tr.render(v)
        fresh.render(v)
        assert torch.equal(tr.img, fresh.img)


@pytest.mark.parametrize("kind", ["fp32", "bf16", "fused"])
def test_narrow_codes_match_oracle(abi, torch, kind):
    """A 3-value code: the zero padding of the code columns 3..7 must not leak in."""
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    sa, ma = synth.with_appearance(sc, mlp, seed=9, A=3)
    sel, w = _pick(sc, 777, 9)
    ref = oracle.decode(sel, w, sa, ma, cams[0])
    got = _decode(abi, torch, sa, ma, cams[0], sel, w, kind, sa.app)
    col = np.abs(got["colors"].astype(np.float64) - ref["colors"]).max()
    assert col <= (2e-5 if kind == "fp32" else 1e-2), col


@pytest.mark.parametrize("bf16", [False, True])
def test_narrow_codes_backward(abi, torch, bf16):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    sa, ma = synth.with_appearance(sc, mlp, seed=10, A=3)
    cam = cams[0]
    rng = np.random.default_rng(6)
    M = 500
    sel = np.sort(rng.choice(sc.N, size=M, replace=False)).astype(np.int64)
    w = rng.uniform(0.05, 1.0, size=M).astype(np.float32)
    G = M * 10
    grads = {k: rng.normal(size=s).astype(np.float32) for k, s in
             (("dmeans", (G, 3)), ("dscales", (G, 3)), ("dquats", (G, 4)), ("dopac", (G,)),
              ("dcolors", (G, 3)))}
    ref = oracle.decode_bwd(sel, w, sa, ma, cam, grads)
    from paper_2403_17898_gb300 import abi as A
    counts = np.zeros(8, np.uint32)
    counts[0], counts[1] = M, G
    drec = np.zeros((G, 9), np.float32)
    drec[:, 5] = grads["dopac"]
    drec[:, 6:9] = grads["dcolors"]
    m, keep = _mlp(ma, sa.app)
    dt = {n: torch.zeros_like(t) for n, t in keep[0].items()}
    dapp = torch.zeros(sc.N, 3, device="cuda")
    scr = torch.empty(abi.decode_bwd_scratch_bytes(M), dtype=torch.uint8, device="cuda")
    abi.decode_bwd(cuda(sa.pos), cuda(sa.feat), cuda(sa.offs), cuda(sa.lv), sc.N, m, cam,
                   cuda(sel.astype(np.int32)), cuda(w), M, cuda(counts.view(np.int32)),
                   cuda(grads["dmeans"]), cuda(grads["dscales"]), cuda(grads["dquats"]),
                   cuda(drec), torch.zeros(sc.N, 32, device="cuda"),
                   torch.zeros(sc.N, 10, 3, device="cuda"), torch.zeros(sc.N, 3, device="cuda"),
                   A.mlp_struct(dt, app=dapp), scr, bf16=bf16)
    torch.cuda.synchronize()
    tol = 6e-2 if bf16 else 1e-4
    for name, got in (("dapp", dapp), ("dw1_app", dt["w1_app"])):
        a, b = got.cpu().numpy(), ref[name]
        assert a.shape == b.shape
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err <= tol, (name, err)
