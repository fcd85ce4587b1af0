"""Frame pipeline over the C ABI: device buffers (torch) and the chain of calls
lod_select -> decode -> project_bin -> sort -> blend_fwd on one CUDA stream.

Only buffer management and call ordering live here; every step runs in ``libogs.so``.
"""
from __future__ import annotations

from dataclasses import dataclass

import math

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
    reserved: int


def _stage(timers, name, st, fn):
    """Runs fn; if ``timers`` is a dict, brackets it with a CUDA event pair on stream st."""
    if timers is None:
        fn()
        return
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    fn()
    e1.record(st)
    timers.setdefault(name, []).append((e0, e1))


# The per-view buffers a view's forward writes and its backward (or the copy of its image)
# reads: pipelined sequences and training steps keep two sets of them, so that the work of
# view v + 1 runs while view v's set is still in use.
_VIEW_KEYS = ("sel_idx", "sel_w", "sel_idx_g", "sel_w_g", "gate_scratch", "dp_scratch", "g",
              "_g_struct", "rec", "depth_key", "rect", "tiles", "pair_gauss", "pair_key", "bins",
              "sort_scratch", "bins_scratch", "counts_t", "img", "T", "n_last", "tile_range",
              "tile_count", "sel_scratch", "active_sel", "active_selw")


class Renderer:
    """Renders views of one anchor set with one decoder at a fixed image size.

    ``sel_cap`` bounds the selected anchors per view and ``pair_cap`` the (tile, Gaussian)
    pairs; ``render(..., check=True)`` grows them and re-renders when a view overflows.
    """

    def __init__(self, scene, mlp, W, H, sel_cap=None, pair_cap=None, k=10, precision="fp32",
                 explicit=None):
        """``explicit``: per-Gaussian attributes (dict log_scale, quat, opacity, color_dc of
        [N][k][...] arrays) for the explicit-Gaussian variant; then ``mlp`` is unused and each
        anchor's k Gaussians come from ogs_explicit_gaussians instead of the decoders."""
        assert precision in ("fp32", "bf16")
        self.precision = precision
        # BF16 neural form: decode and projection in one kernel (ogs_decode_project_bf16);
        # False runs ogs_decode_bf16 and ogs_project_bin as two calls
        self.fuse_decode_project = True
        # BF16 gate: scored inside the selection pass (ogs_lod_select_gated); False runs
        # ogs_lod_select and ogs_proposal_gate_bf16 as two calls
        self.fuse_gate = True
        # inference renders also record each pixel's last blended entry (n_last, which only a
        # backward reads); False skips it in inference mode (training forwards always keep it)
        self.track_last = True
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
        self.explicit = None
        if explicit is not None:
            self.explicit = {n: _cuda(explicit[n], torch.float32) for n in abi.EXPLICIT_NAMES}
            self.mlp = {}
            self._mlp_struct = None
        else:
            self.mlp = {n: _cuda(a, torch.float32) for n, a in zip(names, mlp.arrays())}
        # appearance codes (Sec. 4.4): a code per anchor, seen by the colour decoder
        self.app = None
        if explicit is None and getattr(scene, "app", None) is not None:
            self.app = _cuda(scene.app, torch.float32)
            self.mlp["w1_app"] = _cuda(mlp.w1_app, torch.float32)
        self._structs()
        self.sel_cap = int(sel_cap if sel_cap is not None else max(1024, self.N))
        self.pair_cap = int(pair_cap if pair_cap is not None else 1 << 20)
        # the fused BF16 path's sort places every (tile, Gaussian) pair in its tile's region of
        # tile_cap entries as it counts the pairs, then orders the regions in place
        self.bin_lists = True
        self.tile_cap = 4096
        self._last_binned = False
        self.sel_scratch = torch.empty(abi.lod_select_gated_scratch_bytes(self.N),
                                       dtype=torch.uint8, device="cuda")
        self.counts_t = torch.zeros(8, dtype=torch.int32, device="cuda")
        self.img = torch.empty(3, self.H, self.W, device="cuda")
        self.T = torch.empty(self.H, self.W, device="cuda")
        self.n_last = torch.empty(self.H, self.W, dtype=torch.int32, device="cuda")
        self.tile_range = torch.empty(self.gx * self.gy, 2, dtype=torch.int32, device="cuda")
        self.tile_count = torch.empty(self.gx * self.gy, dtype=torch.int32, device="cuda")
        self._view_set = None            # the second set of per-view buffers, built lazily
        self._view_set_sig = None
        self._view_set_pending = False   # the second set holds views of the last sequence
        self._alloc()

    def _structs(self):
        """(Re)builds the decoder struct after the per-anchor arrays were replaced."""
        if self.explicit is None:
            self._mlp_struct = abi.mlp_struct(self.mlp, k=self.k, app=self.app)

    # -- buffers ---------------------------------------------------------------------------
    def _alloc(self):
        S, G, P = self.sel_cap, self.sel_cap * self.k, self.pair_cap
        dev = "cuda"
        self.sel_idx = torch.empty(S, dtype=torch.int32, device=dev)
        self.sel_w = torch.empty(S, device=dev)
        # gated selection (written by the proposal gate when one is used)
        self.sel_idx_g = torch.empty(S, dtype=torch.int32, device=dev)
        self.sel_w_g = torch.empty(S, device=dev)
        self.gate_scratch = torch.empty(abi.proposal_gate_scratch_bytes(S), dtype=torch.uint8,
                                        device=dev)
        self.dp_scratch = torch.empty(abi.decode_project_scratch_bytes(), dtype=torch.uint8,
                                      device=dev)
        self.g = {"means": torch.empty(G, 3, device=dev), "scales": torch.empty(G, 3, device=dev),
                  "quats": torch.empty(G, 4, device=dev), "opac": torch.empty(G, device=dev),
                  "colors": torch.empty(G, 3, device=dev)}
        self._g_struct = abi.gaussians_struct(self.g)
        self.rec = torch.empty(G, 12, device=dev)
        self.depth_key = torch.empty(G, dtype=torch.int32, device=dev)
        self.rect = torch.empty(G, 2, dtype=torch.int32, device=dev)
        self.tiles = torch.empty(G, dtype=torch.int32, device=dev)
        nt = self.gx * self.gy
        self.pair_gauss = torch.empty(max(P, nt * self.tile_cap, 1), dtype=torch.int32,
                                      device=dev)
        self.pair_key = torch.empty(max(nt * self.tile_cap, 1), dtype=torch.int32, device=dev)
        self.bins = abi.tile_bins(self.pair_key, self.pair_gauss, self.tile_cap)
        self.sort_scratch = torch.empty(abi.sort_scratch_bytes(G, P, nt), dtype=torch.uint8,
                                        device=dev)
        self.bins_scratch = torch.empty(abi.sort_bins_scratch_bytes(nt), dtype=torch.uint8,
                                        device=dev)
        self._grad_bufs_cap = None          # backward buffers follow the capacities

    def _grad_buffers(self):
        """Per-Gaussian backward buffers (record, mean, scale and quaternion gradients) and the
        decoder backward's scratch, sized by the current capacities; allocated on first use."""
        if self._grad_bufs_cap != (self.sel_cap, self.pair_cap):
            G = self.g_cap
            dev = "cuda"
            self.drec = torch.zeros(G, 9, device=dev)
            self.dmeans = torch.empty(G, 3, device=dev)
            self.dscales = torch.empty(G, 3, device=dev)
            self.dquats = torch.empty(G, 4, device=dev)
            self.db_scratch = torch.empty(abi.decode_bwd_scratch_bytes(self.sel_cap),
                                          dtype=torch.uint8, device=dev)
            self._grad_bufs_cap = (self.sel_cap, self.pair_cap)

    @property
    def g_cap(self):
        return self.sel_cap * self.k

    # -- one view --------------------------------------------------------------------------
    def enqueue(self, cam, infer=True, bg=(0.0, 0.0, 0.0), maxc=None, stream=None, timers=None,
                n_eval=None, gate=None, img=None, max_level=None):
        """Enqueues the whole forward pass of one view (no host synchronisation).  If
        ``timers`` is a dict, a CUDA event pair is recorded around every stage under its name
        (on the launching stream).  ``gate = (proposal_weights, p_star)`` inserts the learned
        anchor-visibility gate between selection and decoding.  ``max_level`` caps the octree
        levels the selection may use (levels above it stay inactive: the progressive training
        of Sec. 4.3); the selection then runs as on a tree of max_level + 1 levels."""
        assert int(cam.W) == self.W and int(cam.H) == self.H
        c = abi.camera(cam)
        st = stream if stream is not None else torch.cuda.current_stream()
        # every forward overwrites the per-view buffers a backward reads
        self.generation = getattr(self, "generation", 0) + 1
        self._view_set_pending = False

        def stage(name, fn):
            _stage(timers, name, st, fn)

        fused_gate = gate is not None and self.precision == "bf16" and self.fuse_gate
        if not fused_gate:               # the gated selection resets the counters itself
            with torch.cuda.stream(st):
                self.counts_t.zero_()
        sel, selw = self.sel_idx, self.sel_w
        assert max_level is None or gate is None, "a level cap is a training-time setting"
        NL = self.NL if max_level is None else max(1, min(self.NL, int(max_level) + 1))
        if fused_gate:
            net, p_star = gate
            stage("lod_select", lambda: abi.lod_select_gated(
                self.pos, self.level, self.dL, self.feat, self.N, NL, self.k, c, infer,
                net, p_star, self.sel_idx, self.sel_w, self.sel_cap, self.counts_t,
                self.sel_scratch, st))
        else:
            stage("lod_select", lambda: abi.lod_select(
                self.pos, self.level, self.dL, self.N, NL, self.k, c, infer, self.sel_idx,
                self.sel_w, self.sel_cap, self.counts_t, self.sel_scratch, st))
            if gate is not None:
                net, p_star = gate
                stage("proposal_gate", lambda: abi.proposal_gate(
                    self.pos, self.level, self.feat, self.N, self.NL, self.k, c, net, p_star,
                    self.sel_idx, self.sel_w, self.sel_cap, self.counts_t, self.sel_idx_g,
                    self.sel_w_g, None, self.gate_scratch, st, bf16=self.precision == "bf16"))
                sel, selw = self.sel_idx_g, self.sel_w_g
        self.active_sel, self.active_selw = sel, selw
        fused = self.explicit is None and self.precision == "bf16" and self.fuse_decode_project
        binned = fused and self.bin_lists
        self._last_binned = binned
        if fused:
            # decoded Gaussians go straight to screen records; the Gaussian SoA is written only
            # when a backward pass will need it
            stage("decode_project", lambda: abi.decode_project_bf16(
                self.pos, self.feat, self.offs, self.lv, self.N, self._mlp_struct, c, sel, selw,
                self.sel_cap, self.counts_t, self.rec, self.depth_key, self.rect, self.tiles,
                self.dp_scratch, out=None if infer else self._g_struct,
                tile_count=None if binned else self.tile_count, stream=st))
        else:
            if self.explicit is not None:
                stage("decode", lambda: abi.explicit_gaussians(
                    self.pos, self.offs, self.lv, self.N, self.k, self.explicit, c, sel, selw,
                    self.sel_cap, self.counts_t, self._g_struct, st))
            else:
                dec = abi.decode_bf16 if self.precision == "bf16" else abi.decode
                stage("decode", lambda: dec(
                    self.pos, self.feat, self.offs, self.lv, self.N, self._mlp_struct, c, sel,
                    selw, self.sel_cap, self.counts_t, self._g_struct, st))
            stage("project_bin", lambda: abi.project_bin(
                self._g_struct, self.g_cap, 1, c, self.rec, self.depth_key, self.rect,
                self.tiles, self.counts_t, st, tile_count=self.tile_count))
        if binned:
            stage("sort", lambda: abi.sort_bins(
                self.depth_key, self.rect, self.tiles, self.g_cap, -1, self.gx, self.gy,
                self.bins, self.tile_range, self.counts_t, self.bins_scratch, st))
        else:
            stage("sort", lambda: abi.sort(
                self.depth_key, self.rect, self.tiles, self.g_cap, -1, self.gx, self.gy,
                self.pair_gauss, self.tile_range, self.pair_cap, self.counts_t,
                self.sort_scratch, st, tile_count=self.tile_count))
        n_last = self.n_last if (not infer or self.track_last) else None
        stage("blend_fwd", lambda: abi.blend_fwd(
            self.rec, self.pair_gauss, self.tile_range, self.W, self.H, bg,
            self.img if img is None else img, self.T,
            n_last, sel, self.k, maxc, n_eval, st))

    def backward(self, cam, dimg, grads, dmlp_struct, bg=(0.0, 0.0, 0.0), stream=None,
                 timers=None, on_drec=None):
        """Backward of the view last enqueued (training mode, with ``cam``): dL/dimage ``dimg``
        (f32[3][H][W] on the device) -> ogs_blend_bwd (transmittance recomputed from T_final,
        no per-pair storage) -> ogs_project_bwd -> ogs_decode_bwd (FP32 or tensor-core BF16,
        as the forward) or ogs_explicit_gaussians_bwd.  Anchor gradients accumulate into
        ``grads`` (feat, offs, lv[, app] or offs, lv, ex.*), decoder gradients into the arrays
        of ``dmlp_struct`` (an abi.mlp_struct).  ``on_drec(st)`` runs after the blend backward
        (per-Gaussian statistics read self.drec there)."""
        self._grad_buffers()
        c = abi.camera(cam)
        st = stream if stream is not None else torch.cuda.current_stream()

        def bb():
            with torch.cuda.stream(st):
                self.drec.zero_()
            abi.blend_bwd(self.rec, self.pair_gauss, self.tile_range, self.W, self.H, bg, self.T,
                          self.n_last, dimg, self.drec, st)
        _stage(timers, "blend_bwd", st, bb)
        if on_drec is not None:
            on_drec(st)
        _stage(timers, "project_bwd", st, lambda: abi.project_bwd(
            self._g_struct, self.g_cap, 1, c, self.rect, self.drec, self.dmeans, self.dscales,
            self.dquats, self.counts_t, st))
        sel, selw = self.active_sel, self.active_selw
        if self.explicit is not None:
            gex = {n: grads["ex." + n] for n in abi.EXPLICIT_NAMES}
            _stage(timers, "decode_bwd", st, lambda: abi.explicit_gaussians_bwd(
                self.pos, self.offs, self.lv, self.N, self.k, self.explicit, c, sel, selw,
                self.sel_cap, self.counts_t, self.dmeans, self.dscales, self.dquats, self.drec,
                gex, grads["offs"], grads["lv"], st))
        else:
            _stage(timers, "decode_bwd", st, lambda: abi.decode_bwd(
                self.pos, self.feat, self.offs, self.lv, self.N, self._mlp_struct, c, sel, selw,
                self.sel_cap, self.counts_t, self.dmeans, self.dscales, self.dquats, self.drec,
                grads["feat"], grads["offs"], grads["lv"], dmlp_struct, self.db_scratch, st,
                bf16=self.precision == "bf16"))

    # -- two sets of per-view buffers for pipelined sequences and steps -----------------------
    def _view_snapshot(self):
        return {k: getattr(self, k, None) for k in _VIEW_KEYS}

    @staticmethod
    def _view_signature(d):
        return tuple((k, v.data_ptr(), tuple(v.shape)) for k, v in d.items()
                     if torch.is_tensor(v))

    def _second_view_set(self, d):
        """A set of per-view buffers shaped like ``d`` (the live set)."""
        n = {}
        for k, v in d.items():
            n[k] = torch.empty_like(v) if torch.is_tensor(v) else v
        n["counts_t"] = torch.zeros_like(d["counts_t"])
        n["g"] = {name: torch.empty_like(t) for name, t in d["g"].items()}
        n["_g_struct"] = abi.gaussians_struct(n["g"])
        n["bins"] = abi.tile_bins(n["pair_key"], n["pair_gauss"], self.tile_cap)
        n["active_sel"], n["active_selw"] = None, None
        return n

    def counts(self) -> FrameCounts:
        """Counts of the view last enqueued; after a pipelined sequence or step the overflow
        and timeout flags also cover the views of the second buffer set."""
        v = self.counts_t.cpu().numpy().view(np.uint32)
        c = FrameCounts(*[int(x) for x in v])
        if self._view_set is not None and self._view_set_pending:
            w = self._view_set["counts_t"].cpu().numpy().view(np.uint32)
            c.overflow |= int(w[3])
            c.timeout |= int(w[6])
        return c

    def render_to_host(self, cam, host_img, infer=True, bg=(0.0, 0.0, 0.0), gate=None,
                       zero_copy=True):
        """The end-to-end call: render one view into ``host_img`` (a pinned float32 [3, H, W]
        CPU tensor); returns when the image is on the host.  With ``zero_copy`` the blend
        writes the image straight into the pinned buffer (the device-side image is then not
        updated); otherwise it renders on the device and copies."""
        if zero_copy:
            self.enqueue(cam, infer, bg, gate=gate, img=host_img)
        else:
            self.enqueue(cam, infer, bg, gate=gate)
            host_img.copy_(self.img, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return host_img

    def render_sequence_to_host(self, cams, host_imgs, bg=(0.0, 0.0, 0.0), gate=None,
                                on_frame=None, zero_copy=False):
        """End-to-end rendering of a sequence of views into pinned host memory, pipelined.
        ``host_imgs``: two pinned float32 [3, H, W] CPU tensors used in turn; view i lands in
        ``host_imgs[i % 2]``, and ``on_frame(i, host_img)`` (if given) is called once it is
        there (before that buffer is reused two views later).  By default view i is rendered
        on the device and copied to the host on a copy stream while view i + 1 renders; with
        ``zero_copy`` the blend of view i writes straight into its host buffer instead (no
        copy, but the blend's stores then cross the host link and lengthen it: slower when
        views are pipelined, faster for one view at a time, see render_to_host).  In the
        default form consecutive views also render concurrently, on two compute streams with
        two sets of per-view buffers.  Returns when every image is on the host."""
        if zero_copy:
            done = [None, None]
            for i, cam in enumerate(cams):
                b = i % 2
                if done[b] is not None:
                    done[b].synchronize()            # view i - 2 is on the host
                    if on_frame is not None:
                        on_frame(i - 2, host_imgs[b])
                self.enqueue(cam, True, bg, gate=gate, img=host_imgs[b])
                ev = torch.cuda.Event()
                ev.record()
                done[b] = ev
            for j in range(max(len(cams) - 2, 0), len(cams)):
                b = j % 2
                done[b].synchronize()
                if on_frame is not None:
                    on_frame(j, host_imgs[b])
            return host_imgs
        # two sets of per-view buffers, views alternating between them and between two
        # compute streams: view i + 1 renders while view i is still rendering or being copied
        if getattr(self, "_copy_stream", None) is None:
            self._copy_stream = torch.cuda.Stream()
            self._alt_stream = torch.cuda.Stream()
        comps = (torch.cuda.current_stream(), self._alt_stream)
        live = self._view_snapshot()
        sig = self._view_signature(live)
        if self._view_set is None or self._view_set_sig != sig:
            self._view_set = self._second_view_set(live)
            self._view_set_sig = sig
        sets = [live, self._view_set]
        copied = [None, None]
        try:
            for i, cam in enumerate(cams):
                b = i & 1
                self.__dict__.update(sets[b])
                comp = comps[b]
                if copied[b] is not None:
                    # the set's previous view: its copy must be done before this view's blend
                    # overwrites the device image and before the host buffer is handed out
                    comp.wait_event(copied[b])
                    copied[b].synchronize()
                    if on_frame is not None:
                        on_frame(i - 2, host_imgs[b])
                self.enqueue(cam, True, bg, gate=gate, stream=comp)
                ready = torch.cuda.Event()
                ready.record(comp)
                self._copy_stream.wait_event(ready)
                with torch.cuda.stream(self._copy_stream):
                    host_imgs[b].copy_(self.img, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(self._copy_stream)
                copied[b] = ev
                sets[b] = self._view_snapshot()
            for j in range(max(len(cams) - 2, 0), len(cams)):
                b = j & 1
                copied[b].synchronize()
                if on_frame is not None:
                    on_frame(j, host_imgs[b])
        finally:
            self._view_set = sets[1]
            self.__dict__.update(sets[0])
            comps[0].wait_stream(comps[1])
        self._view_set_pending = len(cams) > 1
        return host_imgs

    def grow_for(self, c):
        """Enlarges the capacities a view overflowed (counts ``c``) and reallocates: the
        selection, and the pair lists (their total, or with per-tile regions the longest
        list, which is what need_pairs reports then)."""
        if c.overflow & 1:
            self.sel_cap = int(c.need_selected * 1.25) + 1024
        if c.overflow & 2:
            if self._last_binned:
                self.tile_cap = int(c.need_pairs * 1.25) + 64
            else:
                self.pair_cap = int(c.need_pairs * 1.25) + 4096
        self._alloc()

    def render(self, cam, infer=True, bg=(0.0, 0.0, 0.0), maxc=None, check=True, gate=None):
        """Renders one view; with ``check`` it synchronises, grows overflowing buffers and
        re-renders until everything fits."""
        for _ in range(4):
            self.enqueue(cam, infer, bg, maxc, gate=gate)
            if not check:
                return None
            c = self.counts()
            if not c.overflow:
                return c
            self.grow_for(c)
            if maxc is not None:
                maxc.zero_()
        raise abi.OgsError("buffers kept overflowing")


def min_count_for(n_views, tau_v):
    """Smallest selection count whose view frequency count / n_views is not below tau_v
    (Sec. 4.2.2: anchors below the threshold are pruned), with the division in float64."""
    c = int(math.ceil(float(tau_v) * n_views))
    while c > 0 and not ((c - 1) / float(n_views) < float(tau_v)):
        c -= 1
    while c / float(n_views) < float(tau_v):
        c += 1
    return c


def progressive_schedule(NL, total, omega):
    """Progressive training (Sec. 4.3): levels 0 .. NL // 2 start active and one more level
    is activated per stage; stage i (finest active level i) lasts N_i iterations with
    N_{i-1} = omega N_i and the N_i summing to `total`.  Returns [(first iteration, level)]."""
    first = NL // 2
    weights = [float(omega) ** (NL - 1 - i) for i in range(first, NL)]
    unit = float(total) / sum(weights)
    out, at = [], 0.0
    for i, w in zip(range(first, NL), weights):
        out.append((int(round(at)), i))
        at += unit * w
    return out


class Trainer(Renderer):
    """One optimisation step over a batch of views: for each view the training-mode forward
    (no next-level anchors), the loss against its target, and the backward chain
    blend_bwd -> project_bwd -> decode_bwd (or the explicit-Gaussian backward) accumulating
    the anchor and decoder gradients; then one Adam update of every trainable array.  With
    ``track_view_frequency`` every training view's selection is counted per anchor, and
    ``prune(tau_v)`` removes the anchors whose view frequency is below tau_v."""

    def __init__(self, scene, mlp, W, H, lr=1e-3, betas=(0.9, 0.999), eps=1e-15, ssim_lambda=0.0,
                 track_view_frequency=False, track_growth=False, track_opacity=False,
                 progressive=None, sparse_adam=True, **kw):
        """``sparse_adam``: the anchor arrays take Adam only on the rows the step's views
        selected (ogs_stamp_selected + ogs_adam_rows: untouched rows keep parameters and
        moments); False updates every row every step.  Decoder weights always update."""
        super().__init__(scene, mlp, W, H, **kw)
        self.ssim_lambda = float(ssim_lambda)   # 0.2 gives the 0.8 L1 + 0.2 D-SSIM loss
        self.lr, self.betas, self.eps = lr, betas, eps
        self.step_count = 0
        self.sparse_adam = bool(sparse_adam)
        dev = "cuda"
        # step number of the last step whose views selected each anchor
        self.stamp = torch.zeros(self.N, dtype=torch.int32, device=dev)
        self.grads = {n: torch.zeros_like(t) for n, t in self._anchor_params().items()}
        self.dmlp = {n: torch.zeros_like(t) for n, t in self.mlp.items()}
        self._structs()
        self.adam_m = {n: torch.zeros_like(t) for n, t in self._anchor_params().items()}
        self.adam_v = {n: torch.zeros_like(t) for n, t in self._anchor_params().items()}
        for n, t in self.mlp.items():
            self.adam_m["mlp." + n] = torch.zeros_like(t)
            self.adam_v["mlp." + n] = torch.zeros_like(t)
        self.dimg = torch.zeros(3, self.H, self.W, device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.loss_scratch = None
        self._ssim_stats = {}            # target data_ptr -> (version, window moments)
        if self.ssim_lambda > 0:
            self.loss_scratch = torch.empty(abi.loss_l1_ssim_scratch_bytes(3, self.H, self.W),
                                            dtype=torch.uint8, device=dev)
        self.track_view_frequency = bool(track_view_frequency)
        self.sel_count = torch.zeros(self.N, dtype=torch.int32, device=dev)
        self.n_views_seen = 0
        # growing statistics (Sec. 4.2.1): per (anchor, slot) sum of the view-space mean
        # gradient norms and the number of views that saw the Gaussian
        self.track_growth = bool(track_growth)
        self._reset_growth_stats()
        # average-opacity statistic (Sec. 4.2.2): per anchor, the summed opacity of its
        # Gaussians and the number of training views that selected it
        self.track_opacity = bool(track_opacity)
        self._reset_opacity_stats()
        # progressive training (Sec. 4.3): (iterations of the progressive stage, omega)
        self.progressive = None
        if progressive is not None:
            total, omega = progressive
            self.progressive = (int(total), progressive_schedule(self.NL, total, omega))
        self._grad_buffers()
        # pipelined steps: the forward of the next view overlaps the backward of this one
        self.pipeline = True
        self._bwd_stream = None

    def _anchor_params(self):
        """Trainable per-anchor arrays: features, offsets and l_v of the neural form; offsets,
        l_v and the explicit attributes of the explicit form."""
        if self.explicit is not None:
            out = {"offs": self.offs, "lv": self.lv}
            out.update({"ex." + n: t for n, t in self.explicit.items()})
            return out
        out = {"feat": self.feat, "offs": self.offs, "lv": self.lv}
        if self.app is not None:
            out["app"] = self.app
        return out

    def _structs(self):
        super()._structs()
        self._dmlp_struct = None
        if self.explicit is None and hasattr(self, "dmlp"):
            self._dmlp_struct = abi.mlp_struct(self.dmlp, k=self.k, app=self.grads.get("app"))

    def _target_stats(self, target, st):
        """The SSIM window moments of a target, computed once per target tensor (recomputed if
        the tensor was modified in place since)."""
        key = target.data_ptr()
        hit = self._ssim_stats.get(key)
        if hit is None or hit[0] != target._version or hit[1].shape[1:] != target.shape:
            stats = torch.empty((2,) + tuple(target.shape), device="cuda")
            abi.ssim_target_stats(target, stats, st)
            hit = (target._version, stats)
            self._ssim_stats[key] = hit
        return hit[1]

    def enqueue(self, cam, infer=True, *args, **kw):
        super().enqueue(cam, infer, *args, **kw)
        if not infer:           # a training view: its anchors take the coming optimiser step
            abi.stamp_selected(self.active_sel, self.counts_t, self.stamp, self.step_count + 1,
                               kw.get("stream"))

    def backward_view(self, cam, target, bg=(0.0, 0.0, 0.0), stream=None, timers=None):
        """Loss and backward of the view last enqueued (its forward must have run in
        training mode with ``cam``); gradients accumulate."""
        st = stream if stream is not None else torch.cuda.current_stream()
        if self.ssim_lambda > 0:
            stats = self._target_stats(target, st)
            _stage(timers, "loss", st, lambda: abi.loss_l1_ssim(
                self.img, target, self.ssim_lambda, self.dimg, self.loss, self.loss_scratch, st,
                target_stats=stats))
        else:
            _stage(timers, "loss", st, lambda: abi.loss_l1(
                self.img, target, self.img.numel(), self.dimg, self.loss, st))
        on_drec = None
        if self.track_growth and self.explicit is None:
            def on_drec(s):
                _stage(timers, "grow_stats", s, lambda: abi.grow_accumulate(
                    self.drec, self.tiles, self.sel_idx, self.counts_t, self.k, self.W, self.H,
                    self.grad_acc, self.grad_cnt, s))
        self.backward(cam, self.dimg, self.grads, self._dmlp_struct, bg, st, timers, on_drec)

    def active_level(self):
        """Finest octree level trained at the current iteration (all levels without a
        progressive schedule, or once its stage is over)."""
        if self.progressive is None:
            return self.NL - 1
        lvl = self.NL - 1
        total, stages = self.progressive
        if self.step_count < total:
            lvl = stages[0][1]
            for first, L in stages:
                if self.step_count >= first:
                    lvl = L
        return lvl

    def in_progressive_stage(self):
        return self.progressive is not None and self.step_count < self.progressive[0]

    def zero_grad(self):
        for t in self.grads.values():
            t.zero_()
        for t in self.dmlp.values():
            t.zero_()

    def optimizer_step(self, stream=None, timers=None):
        self.step_count += 1
        b1, b2 = self.betas
        st = stream if stream is not None else torch.cuda.current_stream()
        pairs = [(t, self.grads[n], n) for n, t in self._anchor_params().items()]
        pairs += [(self.mlp[n], self.dmlp[n], "mlp." + n) for n in self.mlp]

        n_anchor = len(self._anchor_params())

        def run():
            for i, (p, g, n) in enumerate(pairs):
                if self.sparse_adam and i < n_anchor:
                    abi.adam_rows(p, g, self.adam_m[n], self.adam_v[n], self.stamp,
                                  self.step_count, self.lr, b1, b2, self.eps, self.step_count,
                                  True, st)
                else:
                    abi.adam(p, g, self.adam_m[n], self.adam_v[n], p.numel(), self.lr, b1, b2,
                             self.eps, self.step_count, True, st)
        _stage(timers, "adam", st, run)

    def train_step(self, cams, targets, bg=(0.0, 0.0, 0.0), update=True, timers=None):
        """One optimisation step: forward + backward over the views (gradients summed over
        them), then (optionally) the Adam update, which also clears the gradients for the next
        step; returns nothing (the summed per-view loss is left in ``self.loss``)."""
        self.loss.zero_()
        cap = self.active_level() if self.progressive is not None else None
        if not self.pipeline or len(cams) < 2:
            for cam, tgt in zip(cams, targets):
                self._forward_view(cam, bg, timers, cap)
                self.backward_view(cam, tgt, bg, timers=timers)
        else:
            self._pipelined_views(cams, targets, bg, timers, cap)
        if update:
            self.optimizer_step(timers=timers)

    def _forward_view(self, cam, bg, timers, cap):
        self.enqueue(cam, infer=False, bg=bg, timers=timers, max_level=cap)
        if self.track_view_frequency:
            abi.count_selected(self.sel_idx, self.counts_t, self.sel_count)
            self.n_views_seen += 1
        if self.track_opacity:
            abi.opacity_accumulate(self.g["opac"], self.sel_idx, self.counts_t, self.k,
                                   self.opac_sum, self.opac_views)

    def _pipelined_views(self, cams, targets, bg, timers, cap):
        """Views alternate between two sets of per-view buffers.  The forward of each view runs
        on the caller's stream; its loss and backward on a second stream once that forward is
        done, so the next view's forward overlaps them.  A set is reused only after the backward
        that read it has finished; the backward passes run one after another in view order
        (the gradients and the loss accumulate as in the sequential step), and the caller's
        stream waits for the last of them."""
        fwd = torch.cuda.current_stream()
        if self._bwd_stream is None:
            self._bwd_stream = torch.cuda.Stream()
        bwd = self._bwd_stream
        live = self._view_snapshot()
        sig = self._view_signature(live)
        if self._view_set is None or self._view_set_sig != sig:
            self._view_set = self._second_view_set(live)
            self._view_set_sig = sig
        sets = [live, self._view_set]
        done = [None, None]
        try:
            for v, (cam, tgt) in enumerate(zip(cams, targets)):
                i = v & 1
                self.__dict__.update(sets[i])
                if done[i] is not None:
                    fwd.wait_event(done[i])
                self._forward_view(cam, bg, timers, cap)
                ready = torch.cuda.Event()
                ready.record(fwd)
                bwd.wait_event(ready)
                self.backward_view(cam, tgt, bg, stream=bwd, timers=timers)
                done[i] = torch.cuda.Event()
                done[i].record(bwd)
                sets[i] = self._view_snapshot()
            fwd.wait_stream(bwd)
        finally:
            self._view_set = sets[1]
            self.__dict__.update(sets[0])
        self._view_set_pending = True

    def _reset_opacity_stats(self):
        n = self.N if self.track_opacity else 0
        self.opac_sum = torch.zeros(n, device="cuda")
        self.opac_views = torch.zeros(n, dtype=torch.int32, device="cuda")

    def prune_opacity(self, tau_o=0.005):
        """Average-opacity pruning (Sec. 4.2.2): removes the anchors whose Gaussians' average
        opacity over the training views counted since the last prune is below tau_o (anchors
        no counted view selected are kept), compacting every per-anchor array and its
        optimiser state like prune(); clears the opacity statistic.  Returns the kept count."""
        assert self.track_opacity, "opacity pruning needs track_opacity"
        dev = "cuda"
        keep = torch.empty(self.N, dtype=torch.int32, device=dev)
        n_kept = torch.zeros(1, dtype=torch.int32, device=dev)
        scratch = torch.empty(abi.prune_opacity_scratch_bytes(self.N), dtype=torch.uint8,
                              device=dev)
        abi.prune_by_opacity(self.opac_sum, self.opac_views, self.N, self.k, tau_o, keep, n_kept,
                             scratch)
        n = self._compact(keep, n_kept)
        self._reset_opacity_stats()
        return n

    def _reset_growth_stats(self):
        dev = "cuda"
        n = self.N if self.track_growth else 0
        self.grad_acc = torch.zeros(n, self.k, device=dev)
        self.grad_cnt = torch.zeros(n, self.k, dtype=torch.int32, device=dev)

    def grow(self, voxel, tau_g=2e-4, beta=0.2, eps=0.01, next_level=None):
        """Densification step of Sec. 4.2.1 from the statistics accumulated since the last one:
        the LOD-bias update (dL += eps where an anchor's average gradient exceeds 0.25 tau[L]),
        then next-level growing (new anchors in free voxels of level L or L + 1, at the voxel
        centre, l_v = voxel size, zero offsets and LOD bias, features and appearance code of
        the proposing anchor, fresh optimiser state).  ``voxel``: voxel size per level;
        ``next_level`` (default: off during a progressive stage, Sec. 4.3, on otherwise)
        allows the promotion to L + 1.  Clears the statistics; returns the number of anchors
        added."""
        if next_level is None:
            next_level = not self.in_progressive_stage()
        assert self.track_growth and self.explicit is None, "growing needs track_growth"
        dev = "cuda"
        tau, thr_bias = abi.grow_thresholds(tau_g, beta, self.NL)
        abi.update_lod_bias(self.level, self.grad_acc, self.grad_cnt, self.N, self.k, self.NL,
                            thr_bias, eps, self.dL)
        scratch = torch.empty(abi.grow_scratch_bytes(self.N, self.k), dtype=torch.uint8,
                              device=dev)
        n_new = torch.zeros(2, dtype=torch.int32, device=dev)
        max_new = max(1024, self.N // 8)
        while True:
            new_pos = torch.empty(max_new, 3, device=dev)
            new_level = torch.empty(max_new, dtype=torch.uint8, device=dev)
            new_lv = torch.empty(max_new, 3, device=dev)
            parent = torch.empty(max_new, dtype=torch.int32, device=dev)
            abi.grow_anchors(self.pos, self.level, self.offs, self.lv, self.grad_acc,
                             self.grad_cnt, self.N, self.k, self.NL, tau, voxel, new_pos,
                             new_level, new_lv, parent, max_new, n_new, scratch,
                             next_level=next_level)
            got, need = (int(x) for x in n_new.cpu().numpy().view(np.uint32))
            if need <= max_new:
                break
            max_new = need              # the call is deterministic: rerun with room for all
        n = got
        if n:
            def rows(t):
                out = torch.empty((n,) + tuple(t.shape[1:]), dtype=t.dtype, device=dev)
                abi.gather_rows(t, out, t[0].numel() * t.element_size(), parent, None, n)
                return out

            def zeros(t):
                return torch.zeros((n,) + tuple(t.shape[1:]), dtype=t.dtype, device=dev)
            self.pos = torch.cat([self.pos, new_pos[:n]])
            self.level = torch.cat([self.level, new_level[:n]])
            self.dL = torch.cat([self.dL, zeros(self.dL)])
            self.offs = torch.cat([self.offs, zeros(self.offs)])
            self.lv = torch.cat([self.lv, new_lv[:n]])
            self.feat = torch.cat([self.feat, rows(self.feat)])
            if self.app is not None:
                self.app = torch.cat([self.app, rows(self.app)])
            for store in (self.adam_m, self.adam_v):
                for key in list(store):
                    if not key.startswith("mlp."):
                        store[key] = torch.cat([store[key], zeros(store[key])])
            self.sel_count = torch.cat([self.sel_count, zeros(self.sel_count)])
            self.stamp = torch.cat([self.stamp, zeros(self.stamp)])
            if self.track_opacity:
                self.opac_sum = torch.cat([self.opac_sum, zeros(self.opac_sum)])
                self.opac_views = torch.cat([self.opac_views, zeros(self.opac_views)])
            self.N += n
            self.grads = {key: torch.zeros_like(t) for key, t in self._anchor_params().items()}
            self.sel_scratch = torch.empty(abi.lod_select_gated_scratch_bytes(self.N),
                                           dtype=torch.uint8, device=dev)
            self._structs()
        self._reset_growth_stats()
        return n

    def prune(self, tau_v):
        """View-frequency pruning (Sec. 4.2.2): keeps the anchors selected in at least a tau_v
        fraction of the training views counted since the last prune (order preserved), and
        compacts every per-anchor array and its optimiser state.  Returns the kept count."""
        assert self.n_views_seen > 0, "no training views counted"
        dev = "cuda"
        min_count = min_count_for(self.n_views_seen, tau_v)
        keep = torch.empty(self.N, dtype=torch.int32, device=dev)
        n_kept = torch.zeros(1, dtype=torch.int32, device=dev)
        scratch = torch.empty(abi.prune_scratch_bytes(self.N), dtype=torch.uint8, device=dev)
        abi.prune_anchors(self.sel_count, self.N, min_count, keep, n_kept, scratch)
        n = self._compact(keep, n_kept)
        self.sel_count = torch.zeros(self.N, dtype=torch.int32, device=dev)
        self.n_views_seen = 0
        return n

    def _compact(self, keep, n_kept):
        """Keeps the anchors listed in keep[:n_kept] (ascending): every per-anchor array, its
        optimiser state and the per-anchor statistics are gathered on the GPU."""
        dev = "cuda"
        n = int(n_kept.item())

        def gather(t):
            out = torch.empty((n,) + tuple(t.shape[1:]), dtype=t.dtype, device=dev)
            if n:
                row = t[0].numel() * t.element_size()
                abi.gather_rows(t, out, row, keep, n_kept, n)
            return out

        for name in ("pos", "level", "dL", "feat", "offs", "lv"):
            setattr(self, name, gather(getattr(self, name)))
        if self.app is not None:
            self.app = gather(self.app)
        if self.explicit is not None:
            self.explicit = {k: gather(v) for k, v in self.explicit.items()}
        for store in (self.adam_m, self.adam_v):
            for k in list(store):
                if not k.startswith("mlp."):
                    store[k] = gather(store[k])
        self.grads = {k: torch.zeros_like(t) for k, t in self._anchor_params().items()}
        self._structs()
        self.N = n
        self.sel_count = gather(self.sel_count)
        self.stamp = gather(self.stamp)
        self.sel_scratch = torch.empty(abi.lod_select_gated_scratch_bytes(self.N),
                                       dtype=torch.uint8, device=dev)
        if self.track_growth:              # the statistics follow their anchors
            self.grad_acc = gather(self.grad_acc)
            self.grad_cnt = gather(self.grad_cnt)
        if self.track_opacity:
            self.opac_sum = gather(self.opac_sum)
            self.opac_views = gather(self.opac_views)
        return n
