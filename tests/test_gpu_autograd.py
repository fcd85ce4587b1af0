"""The torch.autograd.Function wrappers over the C ABI (RenderFn, PhotometricLossFn,
ProposalFn): gradients reached through ``loss.backward()`` against the FP64 oracle's analytic
gradient, against central finite differences through the GPU forward, and against the direct
backward chain of ``Trainer``."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import cuda, lib_ready

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    return lib_ready()


def _params(rd, torch):
    from paper_2403_17898_gb300.autograd import DECODER_NAMES
    ps = [rd.feat.clone(), rd.offs.clone(), rd.lv.clone()] + \
         [rd.mlp[n].clone() for n in DECODER_NAMES]
    for p in ps:
        p.requires_grad_(True)
    return ps


def _cube():
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    target = np.random.default_rng(1).uniform(size=(3, 128, 128)).astype(np.float32)
    return sc, mlp, cams[0], target


def test_renderfn_gradients_match_oracle(abi):
    """One training view of the 4k-anchor cube, L1 against a seeded target: every gradient
    reached through autograd within the chain tolerance of the oracle's analytic gradient."""
    import torch
    from paper_2403_17898_gb300.autograd import DECODER_NAMES, PhotometricLossFn, RenderFn
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cam, target = _cube()
    rd = Renderer(sc, mlp, 128, 128)
    ps = _params(rd, torch)
    img = RenderFn.apply(rd, cam, (0.0, 0.0, 0.0), *ps)
    loss = PhotometricLossFn.apply(img, cuda(target), 0.0)
    loss.backward()
    fr = oracle.render(sc, mlp, cam, infer=False)
    L, dimg = oracle.l1_loss(fr.out["img"], target)
    assert abs(loss.item() - L) <= 1e-5
    ref = oracle.render_grad(sc, mlp, cam, fr, dimg)
    names = ["dfeat", "doffs", "dlv"] + ["d" + n for n in DECODER_NAMES]
    for name, p in zip(names, ps):
        a, b = p.grad.cpu().numpy(), ref[name]
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err <= 5e-3, (name, err)


def test_renderfn_equals_trainer_chain(abi):
    """The same view through Trainer.backward_view (the benchmark's training step) and through
    autograd: the same kernels, so equal up to the float summation order of the blend
    backward's atomics; also in the BF16 (tensor-core) form."""
    import torch
    from paper_2403_17898_gb300.autograd import DECODER_NAMES, PhotometricLossFn, RenderFn
    from paper_2403_17898_gb300.render import Renderer, Trainer
    sc, mlp, cam, target = _cube()
    for precision in ("fp32", "bf16"):
        tr = Trainer(sc, mlp, 128, 128, precision=precision, ssim_lambda=0.2)
        tr.render(cam, infer=False)
        tr.zero_grad()
        tr.loss.zero_()
        tr.backward_view(cam, cuda(target))
        rd = Renderer(sc, mlp, 128, 128, precision=precision)
        ps = _params(rd, torch)
        img = RenderFn.apply(rd, cam, (0.0, 0.0, 0.0), *ps)
        loss = PhotometricLossFn.apply(img, cuda(target), 0.2)
        loss.backward()
        assert abs(loss.item() - tr.loss.item()) <= 1e-6 * abs(tr.loss.item())
        want = [tr.grads["feat"], tr.grads["offs"], tr.grads["lv"]] + \
               [tr.dmlp[n] for n in DECODER_NAMES]
        for p, w in zip(ps, want):
            a, b = p.grad.cpu().numpy(), w.cpu().numpy()
            assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b) + 1e-12, precision


def test_renderfn_finite_differences(abi):
    """Central differences of the autograd loss through the GPU forward on second-layer
    colour-decoder parameters (they never move an alpha decision and cross no ReLU kink),
    against the autograd gradient."""
    import torch
    from paper_2403_17898_gb300.autograd import PhotometricLossFn, RenderFn
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cam, _ = _cube()
    target = torch.zeros(3, 128, 128, device="cuda")     # L1 = mean intensity: no kink
    rd = Renderer(sc, mlp, 128, 128)
    ps = _params(rd, torch)
    loss = PhotometricLossFn.apply(RenderFn.apply(rd, cam, (0.0, 0.0, 0.0), *ps), target, 0.0)
    loss.backward()
    byname = dict(zip(["feat", "offs", "lv", "w1", "b1", "w2_op", "b2_op", "w2_col", "b2_col",
                       "w2_cov", "b2_cov"], ps))

    def loss_at():
        with torch.no_grad():
            img = RenderFn.apply(rd, cam, (0.0, 0.0, 0.0), *ps)
        return float(img.double().mean().item())

    for name, ix in [("b2_col", (4,)), ("b2_col", (17,)), ("w2_col", (5, 7)),
                     ("w2_col", (22, 30))]:
        p = byname[name]
        g = float(p.grad[ix].item())
        h = 0.02
        with torch.no_grad():
            x0 = float(p[ix].item())
            p[ix] = x0 + h
        lp = loss_at()
        with torch.no_grad():
            p[ix] = x0 - h
        lm = loss_at()
        with torch.no_grad():
            p[ix] = x0
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g) <= 0.03 * abs(g) + 1e-6, (name, ix, g, fd)


def test_renderfn_refuses_stale_backward(abi):
    import torch
    from paper_2403_17898_gb300.abi import OgsError
    from paper_2403_17898_gb300.autograd import PhotometricLossFn, RenderFn
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cam, target = _cube()
    rd = Renderer(sc, mlp, 128, 128)
    ps = _params(rd, torch)
    loss = PhotometricLossFn.apply(RenderFn.apply(rd, cam, (0.0, 0.0, 0.0), *ps),
                                   cuda(target), 0.0)
    rd.render(cam)                       # another view through the same renderer
    with pytest.raises(OgsError):
        loss.backward()


def test_loss_fn_scaled_gradient(abi):
    """PhotometricLossFn: value = the oracle's L1 + D-SSIM; the gradient of 3 x loss is 3 x
    the oracle's gradient (the incoming factor is applied by ogs_scale)."""
    import torch
    from paper_2403_17898_gb300.autograd import PhotometricLossFn
    rng = np.random.default_rng(5)
    img = rng.uniform(size=(3, 37, 53)).astype(np.float32)
    tgt = rng.uniform(size=(3, 37, 53)).astype(np.float32)
    x = cuda(img).requires_grad_(True)
    loss = PhotometricLossFn.apply(x, cuda(tgt), 0.2)
    (3.0 * loss).backward()
    L, g = oracle.photometric_loss(img, tgt, 0.2)
    assert abs(loss.item() - L) <= 1e-5 * abs(L)
    np.testing.assert_allclose(x.grad.cpu().numpy(), 3.0 * g, rtol=1e-4, atol=1e-9)


def test_proposal_fn_matches_oracle(abi):
    """ProposalFn: BCE value and weight gradients of 2 x loss against the oracle's."""
    import torch
    from paper_2403_17898_gb300.autograd import PROPOSAL_NAMES, ProposalFn
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    cam = cams[0]
    net = synth.proposal_mlp(seed=2)
    rd = Renderer(sc, mlp, 128, 128)
    M = 2000
    sel = np.sort(np.random.default_rng(7).choice(sc.N, size=M, replace=False)).astype(np.int64)
    maxc = np.random.default_rng(8).uniform(0, 0.02, size=sc.N).astype(np.float32)
    counts = np.zeros(8, np.uint32)
    counts[0] = M
    ws = [cuda(a).reshape(-1).contiguous() if n == "w3" else cuda(a)
          for n, a in zip(PROPOSAL_NAMES, net.arrays())]
    for w in ws:
        w.requires_grad_(True)
    loss = ProposalFn.apply(rd, cam, cuda(sel.astype(np.int32)), cuda(counts.view(np.int32)),
                            cuda(maxc.view(np.int32)), 0.01, 3.0, *ws)
    (2.0 * loss).backward()
    X = oracle.proposal_inputs(sc.pos, sc.level, sc.feat, sc.NL, sel, cam)
    y = (maxc[sel] >= 0.01).astype(np.float64)
    L, g = oracle.proposal_bce_grad(net, X, y, 3.0)
    assert abs(loss.item() - L) <= 1e-5 * max(1.0, L)
    for n, w in zip(PROPOSAL_NAMES, ws):
        a = w.grad.cpu().numpy().reshape(g[n].shape)
        assert np.linalg.norm(a - 2.0 * g[n]) <= 1e-4 * np.linalg.norm(2.0 * g[n]), n
