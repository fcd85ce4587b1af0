"""Learned anchor-visibility proposal: weights, training on the renderer's own
per-anchor maximum-contribution labels, and evaluation against the plain LOD path.

Orchestration only: scoring, gating, the BCE loss and its gradients run in
``ogs_proposal_gate`` / ``ogs_proposal_train``, the update in ``ogs_adam``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import abi

NAMES = ("w1", "b1", "w2", "b2", "w3", "b3")


class ProposalNet:
    """3-layer MLP (37 -> 64 -> 64 -> 1) on the GPU with its Adam state."""

    def __init__(self, init, lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        self.w = {n: torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()
                  for n, a in zip(NAMES, init.arrays())}
        self.w["w3"] = self.w["w3"].reshape(-1).contiguous()
        self.g = {n: torch.zeros_like(t) for n, t in self.w.items()}
        self.m = {n: torch.zeros_like(t) for n, t in self.w.items()}
        self.v = {n: torch.zeros_like(t) for n, t in self.w.items()}
        self.lr, self.betas, self.eps = lr, betas, eps
        self.steps = 0
        self.scratch = torch.empty(abi.proposal_train_scratch_bytes(), dtype=torch.uint8,
                                   device="cuda")
        self.loss = torch.zeros(1, device="cuda")

    def numpy(self):
        """Weights as float32 arrays in the synth.ProposalMLP layout."""
        out = {n: t.detach().cpu().numpy() for n, t in self.w.items()}
        out["w3"] = out["w3"].reshape(1, -1)
        return out

    def train_view(self, rd, cam, sel_idx, counts, maxc, tau, pos_weight=1.0):
        abi.proposal_train(rd.pos, rd.level, rd.feat, rd.N, rd.NL, cam, self.w, sel_idx, counts,
                           maxc, tau, self.g, self.loss, self.scratch, pos_weight)

    def step(self):
        self.steps += 1
        b1, b2 = self.betas
        for n in NAMES:
            abi.adam(self.w[n], self.g[n], self.m[n], self.v[n], self.w[n].numel(), self.lr, b1,
                     b2, self.eps, self.steps, True)


@dataclass
class ViewLabels:
    cam: object
    sel_idx: torch.Tensor
    counts: torch.Tensor
    maxc: torch.Tensor
    n_selected: int = 0


def collect_labels(rd, cams, infer=True):
    """Renders every view with the plain LOD path and keeps its selection and per-anchor
    maximum contribution (the training labels)."""
    out = []
    for cam in cams:
        maxc = torch.zeros(rd.N, dtype=torch.int32, device="cuda")
        c = rd.render(cam, infer=infer, maxc=maxc)
        out.append(ViewLabels(cam, rd.sel_idx.clone(), rd.counts_t.clone(), maxc, c.n_selected))
    return out


def train(net, rd, views, epochs=20, tau=1.0 / 255.0, seed=0, pos_weight=1.0):
    """Adam on the mean (weighted) BCE of each view's selected anchors, views shuffled per
    epoch; returns the mean loss per epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    for _ in range(epochs):
        net.loss.zero_()
        for i in rng.permutation(len(views)):
            v = views[i]
            net.train_view(rd, v.cam, v.sel_idx, v.counts, v.maxc, tau, pos_weight)
            net.step()
        hist.append(float(net.loss.item()) / len(views))
    return hist


def psnr(a, b):
    mse = float(torch.mean((a.float() - b.float()) ** 2).item())
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)


def full_detail(cam):
    """Same pose with every level selected (L* clamps at its maximum): the stand-in ground
    truth that the plain and gated paths are both compared with."""
    import copy
    c = copy.copy(cam)
    c.s = 1e-6
    return c


@dataclass
class GateAssessment:
    """Image cost of the gated form on a set of views against full-detail renders."""
    pooled_db: float              # 10 log10(sum MSE gated / sum MSE plain) over the views
    psnr_plain: list              # per view: PSNR of the plain path vs full detail (dB)
    psnr_gated: list              # per view: PSNR of the gated path vs full detail (dB)
    kept: list                    # per view: gated / plain selected anchors

    @property
    def dpsnr(self):
        return [a - b for a, b in zip(self.psnr_plain, self.psnr_gated)]


def assess(rd, full_rd, cams, gate, plain_precision="fp32", gate_precision="bf16"):
    """Renders every view three ways: full detail (every level, ``full_rd``), the plain LOD
    path (``plain_precision``, no gate) and the gated path (``gate_precision`` with
    ``gate = (weights, p_star)``); returns the pooled and per-view PSNR figures."""
    se_plain = se_gate = 0.0
    pp, pg, kept = [], [], []
    prec = rd.precision
    try:
        for cam in cams:
            full_rd.render(full_detail(cam))
            ref = full_rd.img
            rd.precision = plain_precision
            c0 = rd.render(cam)
            plain = rd.img.clone()
            rd.precision = gate_precision
            c1 = rd.render(cam, gate=gate)
            se_plain += float(torch.mean((plain - ref) ** 2).item())
            se_gate += float(torch.mean((rd.img - ref) ** 2).item())
            pp.append(psnr(plain, ref))
            pg.append(psnr(rd.img, ref))
            kept.append(c1.n_selected / max(c0.n_selected, 1))
    finally:
        rd.precision = prec
    pooled = 10.0 * math.log10(se_gate / se_plain) if se_plain > 0 else 0.0
    return GateAssessment(pooled, pp, pg, kept)


CANDIDATES = (0.001, 0.002, 0.005, 0.01, 0.02, 0.05, 0.1, 0.2, 0.3, 0.5, 0.6, 0.7, 0.8, 0.9,
              0.95)


def calibrate(rd, full_rd, cams, weights, budget_db, candidates=CANDIDATES, **kw):
    """Largest threshold p* among ``candidates`` whose pooled PSNR loss on ``cams`` (views
    the network was trained on, never the views it is judged on) is within ``budget_db``;
    0 if none is.  Returns (p_star, [(p*, pooled dB, median dB, max dB, kept fraction)]);
    ``kw`` (precisions) goes to ``assess``."""
    p_star, curve = 0.0, []
    for cand in candidates:
        a = assess(rd, full_rd, cams, (weights, cand), **kw)
        curve.append((cand, a.pooled_db, float(np.median(a.dpsnr)), float(np.max(a.dpsnr)),
                      float(np.mean(a.kept))))
        if a.pooled_db <= budget_db:
            p_star = cand
    return p_star, curve
