"""Frame pipeline over the C ABI: device buffers (torch) and the chain of calls
lod_select -> decode -> project_bin -> sort -> blend_fwd on one CUDA stream.

Only buffer management and call ordering live here; every step runs in ``libogs.so``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import abi

TILE = 16


def _cuda(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


@dataclass
class FrameCounts:
    n_selected: int
    n_gaussians: int
    n_pairs: int
    overflow: int
    need_selected: int
    need_pairs: int
    timeout: int
    n_visible: int


class Renderer:
    """Renders views of one anchor set with one decoder at a fixed image size.

    ``sel_cap`` bounds the selected anchors per view and ``pair_cap`` the (tile, Gaussian)
    pairs; ``render(..., check=True)`` grows them and re-renders when a view overflows.
    """

    def __init__(self, scene, mlp, W, H, sel_cap=None, pair_cap=None, k=10):
        self.k = k
        self.W, self.H = int(W), int(H)
        self.gx, self.gy = (self.W + TILE - 1) // TILE, (self.H + TILE - 1) // TILE
        self.N = int(scene.pos.shape[0])
        self.NL = int(scene.NL)
        self.pos = _cuda(scene.pos, torch.float32)
        self.level = _cuda(scene.level, torch.uint8)
        self.dL = _cuda(scene.dL, torch.float32)
        self.feat = _cuda(scene.feat, torch.float32)
        self.offs = _cuda(scene.offs, torch.float32)
        self.lv = _cuda(scene.lv, torch.float32)
        names = ("w1", "b1", "w2_op", "b2_op", "w2_col", "b2_col", "w2_cov", "b2_cov")
        self.mlp = {n: _cuda(a, torch.float32) for n, a in zip(names, mlp.arrays())}
        self._mlp_struct = abi.mlp_struct(self.mlp, k=k)
        self.sel_cap = int(sel_cap if sel_cap is not None else max(1024, self.N))
        self.pair_cap = int(pair_cap if pair_cap is not None else 1 << 20)
        self.sel_scratch = torch.empty(abi.lod_select_scratch_bytes(self.N), dtype=torch.uint8,
                                       device="cuda")
        self.counts_t = torch.zeros(8, dtype=torch.int32, device="cuda")
        self.img = torch.empty(3, self.H, self.W, device="cuda")
        self.T = torch.empty(self.H, self.W, device="cuda")
        self.n_last = torch.empty(self.H, self.W, dtype=torch.int32, device="cuda")
        self.tile_range = torch.empty(self.gx * self.gy, 2, dtype=torch.int32, device="cuda")
        self._alloc()

    # -- buffers ---------------------------------------------------------------------------
    def _alloc(self):
        S, G, P = self.sel_cap, self.sel_cap * self.k, self.pair_cap
        dev = "cuda"
        self.sel_idx = torch.empty(S, dtype=torch.int32, device=dev)
        self.sel_w = torch.empty(S, device=dev)
        self.g = {"means": torch.empty(G, 3, device=dev), "scales": torch.empty(G, 3, device=dev),
                  "quats": torch.empty(G, 4, device=dev), "opac": torch.empty(G, device=dev),
                  "colors": torch.empty(G, 3, device=dev)}
        self._g_struct = abi.gaussians_struct(self.g)
        self.rec = torch.empty(G, 12, device=dev)
        self.depth_key = torch.empty(G, dtype=torch.int32, device=dev)
        self.rect = torch.empty(G, 2, dtype=torch.int32, device=dev)
        self.tiles = torch.empty(G, dtype=torch.int32, device=dev)
        self.pair_gauss = torch.empty(max(P, 1), dtype=torch.int32, device=dev)
        self.sort_scratch = torch.empty(abi.sort_scratch_bytes(G, P, self.gx * self.gy),
                                        dtype=torch.uint8, device=dev)

    @property
    def g_cap(self):
        return self.sel_cap * self.k

    # -- one view --------------------------------------------------------------------------
    def enqueue(self, cam, infer=True, bg=(0.0, 0.0, 0.0), maxc=None, stream=None):
        """Enqueues the whole forward pass of one view (no host synchronisation)."""
        assert int(cam.W) == self.W and int(cam.H) == self.H
        c = abi.camera(cam)
        self.counts_t.zero_()
        abi.lod_select(self.pos, self.level, self.dL, self.N, self.NL, self.k, c, infer,
                       self.sel_idx, self.sel_w, self.sel_cap, self.counts_t, self.sel_scratch,
                       stream)
        abi.decode(self.pos, self.feat, self.offs, self.lv, self.N, self._mlp_struct, c,
                   self.sel_idx, self.sel_w, self.sel_cap, self.counts_t, self._g_struct, stream)
        abi.project_bin(self._g_struct, self.g_cap, 1, c, self.rec, self.depth_key, self.rect,
                        self.tiles, self.counts_t, stream)
        abi.sort(self.depth_key, self.rect, self.tiles, self.g_cap, -1, self.gx, self.gy,
                 self.pair_gauss, self.tile_range, self.pair_cap, self.counts_t,
                 self.sort_scratch, stream)
        abi.blend_fwd(self.rec, self.pair_gauss, self.tile_range, self.W, self.H, bg, self.img,
                      self.T, self.n_last, self.sel_idx, self.k, maxc, stream)

    def counts(self) -> FrameCounts:
        v = self.counts_t.cpu().numpy().view(np.uint32)
        return FrameCounts(*[int(x) for x in v])

    def render(self, cam, infer=True, bg=(0.0, 0.0, 0.0), maxc=None, check=True):
        """Renders one view; with ``check`` it synchronises, grows overflowing buffers and
        re-renders until everything fits."""
        for _ in range(4):
            self.enqueue(cam, infer, bg, maxc)
            if not check:
                return None
            c = self.counts()
            if not c.overflow:
                return c
            if c.overflow & 1:
                self.sel_cap = int(c.need_selected * 1.25) + 1024
            if c.overflow & 2:
                self.pair_cap = int(c.need_pairs * 1.25) + 4096
            self._alloc()
            if maxc is not None:
                maxc.zero_()
        raise abi.OgsError("buffers kept overflowing")
