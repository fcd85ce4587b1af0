"""``torch.autograd.Function`` wrappers over the C ABI, so that the renderer's hand-written
backward is reachable from ordinary PyTorch code:

    img  = RenderFn.apply(rd, cam, bg, feat, offs, lv, *decoder_weights)     # one view
    loss = PhotometricLossFn.apply(img, target, 0.2)                          # Sec. 5.1.5
    loss.backward()                     # blend_bwd -> project_bwd -> decode_bwd, in libogs
    bce  = ProposalFn.apply(rd, net_weights..., cam, sel_idx, counts, maxc, tau, pos_weight)

Only argument marshalling happens here: every forward and backward step runs in the library's
kernels (the chain-rule factor a loss receives is applied by ``ogs_scale`` or, for the
proposal, by ``ogs_proposal_train``'s ``dloss`` argument).
"""
from __future__ import annotations

import torch

from . import abi

DECODER_NAMES = ("w1", "b1", "w2_op", "b2_op", "w2_col", "b2_col", "w2_cov", "b2_cov")
PROPOSAL_NAMES = ("w1", "b1", "w2", "b2", "w3", "b3")


def _plain(t, name):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise abi.OgsError(f"{name}: expected a contiguous float32 CUDA tensor")
    return t.detach()


class RenderFn(torch.autograd.Function):
    """One view through the training-mode forward (Sec. 4.1.3 selection without next-level
    anchors, Sec. 3.2 decoding, Sec. 3.1 projection, tile lists and blending, Eq. 2) of a
    ``render.Renderer``; the backward is the library's analytic chain (the blend backward
    recovers each pixel's transmittance from T_final by division instead of storing it).

    apply(rd, cam, bg, feat, offs, lv, w1, b1, w2_op, b2_op, w2_col, b2_col, w2_cov, b2_cov)
    -> image f32[3][H][W] (a new tensor per call).

    The trainable arrays passed in are the ones the kernels read (the renderer is re-bound to
    them); anchor positions, levels and LOD biases stay the renderer's constants.  The
    renderer's per-view buffers hold one view: run the backward of a view before the next
    forward through the same renderer (checked), or use one renderer per view in flight.
    The forward synchronises once to grow the renderer's buffers if the view overflows them.
    """

    @staticmethod
    def forward(ctx, rd, cam, bg, feat, offs, lv, *weights):
        if rd.explicit is not None:
            raise abi.OgsError("RenderFn drives the neural-Gaussian form")
        if len(weights) != len(DECODER_NAMES):
            raise abi.OgsError("RenderFn expects the eight decoder arrays")
        rd.feat = _plain(feat, "feat")
        rd.offs = _plain(offs, "offs")
        rd.lv = _plain(lv, "lv")
        for n, w in zip(DECODER_NAMES, weights):
            rd.mlp[n] = _plain(w, n)
        rd._structs()
        img = torch.empty(3, rd.H, rd.W, device="cuda")
        for _ in range(4):
            rd.enqueue(cam, infer=False, bg=bg, img=img)
            c = rd.counts()
            if not c.overflow:
                break
            rd.grow_for(c)
        else:
            raise abi.OgsError("buffers kept overflowing")
        ctx.rd, ctx.cam, ctx.bg, ctx.generation = rd, cam, tuple(bg), rd.generation
        ctx.shapes = [t.shape for t in (feat, offs, lv) + tuple(weights)]
        return img

    @staticmethod
    def backward(ctx, dimg):
        rd = ctx.rd
        if rd.generation != ctx.generation:
            raise abi.OgsError("the renderer rendered another view since this forward: run "
                               "each view's backward before the next forward")
        dimg = dimg.contiguous()
        z = [torch.zeros(s, device="cuda") for s in ctx.shapes]
        grads = {"feat": z[0], "offs": z[1], "lv": z[2]}
        dmlp = dict(zip(DECODER_NAMES, z[3:]))
        rd.backward(ctx.cam, dimg, grads, abi.mlp_struct(dmlp, k=rd.k), ctx.bg)
        return (None, None, None, *z)


class PhotometricLossFn(torch.autograd.Function):
    """Sec. 5.1.5 photometric loss (1 - lambda) L1 + lambda D-SSIM of one image against its
    target (lambda = 0 gives the mean L1), value and gradient from ``ogs_loss_l1`` /
    ``ogs_loss_l1_ssim``.  apply(img, target, lam) -> 1-element loss tensor."""

    @staticmethod
    def forward(ctx, img, target, lam):
        img, target = _plain(img, "img"), _plain(target, "target")
        dimg = torch.empty_like(img)
        loss = torch.zeros(1, device="cuda")
        if lam > 0:
            C, H, W = img.shape
            scr = torch.empty(abi.loss_l1_ssim_scratch_bytes(C, H, W), dtype=torch.uint8,
                              device="cuda")
            abi.loss_l1_ssim(img, target, lam, dimg, loss, scr)
        else:
            abi.loss_l1(img, target, img.numel(), dimg, loss)
        ctx.save_for_backward(dimg)
        return loss

    @staticmethod
    def backward(ctx, dloss):
        (dimg,) = ctx.saved_tensors
        abi.scale(dimg, dloss.contiguous())
        return dimg, None, None


class ProposalFn(torch.autograd.Function):
    """Training objective of the learned anchor-visibility proposal: mean weighted binary
    cross-entropy of its keep probability over one view's selected anchors against the
    renderer's own labels (the anchor's largest T alpha >= tau), value and weight gradients
    from ``ogs_proposal_train`` (the incoming gradient enters as its ``dloss``).

    apply(rd, cam, sel_idx, counts, maxc, tau, pos_weight, w1, b1, w2, b2, w3, b3)
    -> 1-element loss tensor.  ``rd`` supplies the anchor arrays; sel_idx / counts / maxc are
    a view's selection, its counters and its max-contribution labels (proposal.ViewLabels)."""

    @staticmethod
    def forward(ctx, rd, cam, sel_idx, counts, maxc, tau, pos_weight, *weights):
        if len(weights) != len(PROPOSAL_NAMES):
            raise abi.OgsError("ProposalFn expects the six network arrays")
        w = {n: _plain(t, n) for n, t in zip(PROPOSAL_NAMES, weights)}
        loss = torch.zeros(1, device="cuda")
        ctx.args = (rd, cam, sel_idx, counts, maxc, float(tau), float(pos_weight), w)
        ctx.shapes = [t.shape for t in weights]
        g = {n: torch.zeros_like(t) for n, t in w.items()}
        scr = torch.empty(abi.proposal_train_scratch_bytes(), dtype=torch.uint8, device="cuda")
        abi.proposal_train(rd.pos, rd.level, rd.feat, rd.N, rd.NL, cam, w, sel_idx, counts,
                           maxc, tau, g, loss, scr, pos_weight)
        return loss

    @staticmethod
    def backward(ctx, dloss):
        rd, cam, sel_idx, counts, maxc, tau, pos_weight, w = ctx.args
        g = {n: torch.zeros_like(t) for n, t in w.items()}
        scr = torch.empty(abi.proposal_train_scratch_bytes(), dtype=torch.uint8, device="cuda")
        abi.proposal_train(rd.pos, rd.level, rd.feat, rd.N, rd.NL, cam, w, sel_idx, counts,
                           maxc, tau, g, None, scr, pos_weight, dloss=dloss.contiguous())
        return (None,) * 7 + tuple(g[n] for n in PROPOSAL_NAMES)
