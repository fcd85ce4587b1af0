#!/usr/bin/env python
"""Benchmark: 1080p frames/s of the Octree-GS LOD renderer hot path on GB300.

Workload (default): 2M anchors over 8 octree levels on a 2 km synthetic city grid, k = 10
neural Gaussians per anchor, 1920x1080, a 120-pose zoom-out from 10 m to 2 km altitude.  A
step is one view through the whole forward hot path (LOD selection, learned visibility gate,
BF16 tensor-core decoding, projection and binning, sorting, blending); step i renders pose
(rank + i * world) mod 120.  The same steps are also timed on the plain FP32 path (no gate,
FP32 decode), and the gate's image cost is assessed on 60 held-out poses.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on the host
cores instead (rank 0 only), each step a 1/16 sub-view of a frame.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "city2M_1080p"
WORKLOAD_DESC = ("2M anchors / 8 levels / 2 km synthetic city grid, k=10, 1920x1080, "
                 "120-pose zoom-out 10 m -> 2 km, FP32 decode")
METRIC = "1080p FPS (frames/s)"
# FP32 operations of one (pixel, Gaussian) blend evaluation of Eq. 2 with the rasterizer
# conventions (one ex2 and about fifteen FP32 operations: offset, quadratic form, skip and
# clamp tests, transmittance and stop, weight and colour), counted over the tests the kernel
# executes (its n_eval output)
OPS_PER_EVAL = 16
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:8]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = set()
        for _, _, flags in rows:
            for n, v in zip(names[1:], flags[1:]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload():
    import synth
    return synth.CONFIGS[WORKLOAD]()


def pose_of(rank, ws, n_poses):
    """Pose of step i on this rank: ranks interleave over the path (weak scaling: every rank
    renders its own frames, no data exchange)."""
    return lambda i: (rank + i * ws) % n_poses


def max_over_ranks(values, ws, device):
    """Element-wise maximum of per-rank timings (the job takes as long as its slowest rank)."""
    if ws <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


# ---------------------------------------------------------------------------------------
# algorithmic bytes per stage (inputs read once, outputs written once)
# ---------------------------------------------------------------------------------------

def stage_bytes(N, M, G, P, n_tiles, pixels, k=10):
    return {
        "lod_select": N * (12 + 1 + 4) + M * 8,
        "decode": M * (8 + 12 + 128 + 12 * k + 12) + G * 56,
        "project_bin": G * 56 + G * (48 + 4 + 8 + 4),
        "decode_project": M * (8 + 12 + 128 + 12 * k + 12) + G * (48 + 4 + 8 + 4),
        "sort": G * (4 + 8 + 4) + P * 4 + n_tiles * 8,
        "blend_fwd": P * (36 + 4) + n_tiles * 8 + pixels * (12 + 4 + 4),
    }


# ---------------------------------------------------------------------------------------
# CPU oracle timing
# ---------------------------------------------------------------------------------------

def oracle_frame(sc, mlp, cam):
    import oracle
    oracle.render(sc, mlp, cam, infer=True)


def sub_view(cam, i, nx=4, ny=4):
    """Camera for the i-th of nx*ny windows of a frame: same centre and focal length, optical
    axis through the window centre, window-sized image."""
    import synth
    W, H = cam.W // nx, cam.H // ny
    wx, wy = i % nx, i // nx
    u = (wx + 0.5) * W - 0.5
    v = (wy + 0.5) * H - 0.5
    d_cam = np.array([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, 1.0])
    d_world = cam.R.astype(np.float64).T @ d_cam
    c = cam.campos.astype(np.float64)
    up = -cam.R[1].astype(np.float64)
    sv = synth.look_at_camera(c, c + d_world, W, H, up=tuple(up), d_max=cam.d_max)
    sv.fx = sv.fy = float(np.float32(cam.fx))
    return sv


def cpu_baseline(sc, mlp, cams, frames=8):
    idx = np.linspace(0, len(cams) - 1, frames).round().astype(int)
    oracle_frame(sc, mlp, cams[int(idx[0])])          # builds the library, warms caches
    t0 = time.perf_counter()
    for i in idx:
        oracle_frame(sc, mlp, cams[int(i)])
    dt = time.perf_counter() - t0
    return {"value": frames / dt, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{frames} full 1920x1080 frames at poses {idx.tolist()} of the "
                      f"120-pose path ({dt:.1f} s, FP64 C oracle, OpenMP in blending)"}


SINGLE_THREAD_POSES = (30, 90)


def run_cpu_single(args):
    """Times the oracle on one host thread (launched by the GPU arm with OMP_NUM_THREADS=1):
    full 1080p frames of the city path; prints one JSON line."""
    sc, mlp, cams = _workload()
    sc, mlp = _as_f64(sc, mlp)
    oracle_frame(sc, mlp, cams[0])
    t0 = time.perf_counter()
    for p in SINGLE_THREAD_POSES:
        oracle_frame(sc, mlp, cams[p])
    dt = time.perf_counter() - t0
    print(json.dumps({"value": len(SINGLE_THREAD_POSES) / dt, "unit": "frames/s", "cores": 1,
                      "s_per_frame": dt / len(SINGLE_THREAD_POSES),
                      "sample": f"{len(SINGLE_THREAD_POSES)} full 1920x1080 frames at poses "
                                f"{list(SINGLE_THREAD_POSES)} ({dt:.1f} s, one thread)"}))
    return 0


def cpu_baseline_single_thread():
    """The oracle on one host thread, in a child process (the OpenMP thread count is fixed
    when the oracle library loads)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-single"], env=env,
                       capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline_train_view():
    """One view of the batched training step (8M anchors, 10 levels, 1080p, L1 + D-SSIM) on
    the oracle with every host core: training-mode forward, loss and analytic backward; a step
    of 16 views is extrapolated x16."""
    import oracle
    import synth
    sc, mlp, cams = synth.CONFIGS["city8M_1080p"]()
    pose = 20                            # the 6th of the step's 16 views (every 4th pose)
    cam = cams[pose]
    target = np.random.default_rng(4).uniform(size=(3, cam.H, cam.W))
    t0 = time.perf_counter()
    fr = oracle.render(sc, mlp, cam, infer=False)
    L, dimg = oracle.photometric_loss(fr.out["img"], target, 0.2)
    oracle.render_grad(sc, mlp, cam, fr, dimg)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / (16.0 * dt), "unit": "train-steps/s", "cores": os.cpu_count(),
            "s_per_view": dt, "s_per_step_x16": 16.0 * dt, "kind": "oracle",
            "sample": f"one of the 16 training views of a step (8M anchors, 1920x1080, pose "
                      f"{pose}), forward + L1/D-SSIM + backward in FP64, {dt:.1f} s; the step "
                      f"time is 16x that"}


def _as_f64(sc, mlp):
    """One-time float64 copies so the oracle's per-call conversions are no-ops."""
    import synth
    sc64 = synth.Scene(pos=sc.pos.astype(np.float64), level=sc.level.astype(np.int32),
                       dL=sc.dL.astype(np.float64), feat=sc.feat.astype(np.float64),
                       offs=sc.offs.astype(np.float64), lv=sc.lv.astype(np.float64),
                       NL=sc.NL, k=sc.k, meta=sc.meta)
    mlp64 = synth.DecoderMLP(*[a.astype(np.float64) for a in mlp.arrays()])
    return sc64, mlp64


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    sc, mlp, cams = _workload()
    sc, mlp = _as_f64(sc, mlp)
    n = len(cams)
    views = lambda step: sub_view(cams[(step // 16) % n], step % 16)
    oracle_frame(sc, mlp, views(0))
    for s in range(args.warmup):
        oracle_frame(sc, mlp, views(s))
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle_frame(sc, mlp, views(args.warmup + s))
    dt = time.perf_counter() - t0
    fps = (args.steps / 16.0) / dt
    sample = ("each step renders one 480x270 sub-view (1/16 of the pixels, same focal length, "
              "axis through the window centre) of a 1080p frame; 16 steps = 1 frame")
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC},
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

# kernels each ABI call launches per frame (the timed form: fused BF16 decode + projection,
# then ogs_sort_bins: bin_regions, bin_deferred, bins_scan, tile_sort_warp, tile_sort_listed)
LAUNCHES = {"lod_select": 2, "lod_select_gated": 3, "decode_project": 2, "sort": 5,
            "blend_fwd": 1}
DPSNR_GATE_DB = 0.05
# DRAM bytes (read + write) of one blend_fwd launch and its issue-slot use, from an ncu
# capture of the same kernel on this workload (pose 14 of the path, BF16 decode)
BLEND_FWD_DRAM_BYTES = 33.09e6
BLEND_FWD_ISSUE_FRAC = 0.83
BLEND_FWD_TRAFFIC_NOTE = ("dram read + write bytes of one launch (pose 14, the no-n_last "
                          "variant the timed frames run) from ncu: 31.72 MB read, 1.38 MB "
                          "written; the records written by the projection mostly stay in L2")


def _time_form(rd, cams, pose, steps, warmup, gate, flush, clk_index):
    """Device time of `steps` frames (a CUDA event pair per frame, L2 flushed between frames)
    and the clocks seen meanwhile; then the mean time of every stage from a second pass over
    the same poses with an event pair around each stage.  The stage events sit between the
    frame's kernels and break their launch chaining, so the frame time is taken without them."""
    import torch
    for i in range(warmup):
        flush.zero_()
        rd.enqueue(cams[pose(i)], gate=gate)
    torch.cuda.synchronize()
    steps_ev = []
    with ClockSampler(clk_index) as clk:
        torch.cuda.synchronize()
        for i in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rd.enqueue(cams[pose(warmup + i)], gate=gate)
            e1.record()
            steps_ev.append((e0, e1))
        torch.cuda.synchronize()
    c = rd.counts()
    assert c.overflow == 0 and c.timeout == 0, "overflow or expired wait in timed steps"
    step_ms = [a.elapsed_time(b) for a, b in steps_ev]
    timers = {}
    for i in range(min(steps, 300)):
        flush.zero_()
        rd.enqueue(cams[pose(warmup + i)], timers=timers, gate=gate)
    torch.cuda.synchronize()
    stage_ms = {k: float(np.mean([a.elapsed_time(b) for a, b in v])) for k, v in timers.items()}
    return sum(step_ms) / 1e3, stage_ms, clk.summary()


def _per_pose(rd, cams, gate=None):
    """Selected anchors, Gaussians, pairs and blend evaluations of every pose (untimed)."""
    import torch
    n_eval = torch.zeros(rd.H, rd.W, dtype=torch.int32, device="cuda")
    out = []
    for cam in cams:
        c = rd.render(cam, gate=gate)
        rd.enqueue(cam, n_eval=n_eval, gate=gate)
        out.append((c.n_selected, c.n_gaussians, c.n_pairs, int(n_eval.sum().item())))
    return out


# training-step workloads: (scene, views per step, SSIM weight, timed steps, warm-up steps)
TRAIN_WORKLOADS = (
    ("city8M_1080p", 16, 0.2, 8, 3,
     "8M anchors / 10 levels / 4 km city grid, 16 views of 1920x1080 per step (every 4th pose "
     "of a 64-pose zoom-out 8 m -> 4 km), 0.8 L1 + 0.2 D-SSIM, dense Adam over all anchors "
     "and decoder weights; targets: the views rendered before N(0, 0.05) noise was added to "
     "the anchor features"),
    ("street500k_1600x900", 1, 0.0, 60, 5,
     "500k anchors / 6 levels / 600 m street grid, one 1600x900 view per step (30-pose "
     "zoom-out 8 m -> 250 m, cycled), L1, dense Adam; targets: the views rendered before "
     "N(0, 0.05) noise was added to the anchor features"),
)


PRUNE_TAU_V = 0.01          # the paper's visibility threshold for large-scale scenes
PRUNE_TAU_O = 0.005         # average-opacity threshold (the paper gives none: Scaffold-GS's)
GROW_TAU_G, GROW_BETA, GROW_EPS = 2e-4, 0.2, 0.01   # the paper's growing defaults


def _explicit_bench(cams, pose, steps, warmup, flush, clk_index):
    """1080p frames/s of the explicit-Gaussian variant (each anchor's k Gaussians carry their
    own attributes, no decoders) on the same scene and path; the rest of the path is shared."""
    import torch
    import synth
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, _ = _workload()
    attr = synth.explicit_attributes(sc, seed=0)
    W, H = cams[0].W, cams[0].H
    rd = Renderer(sc, None, W, H, sel_cap=200_000, pair_cap=6_000_000, explicit=attr)
    rd.track_last = False
    for cam in cams:                      # size the buffers on every pose
        rd.render(cam)
    t, stages, clk = _time_form(rd, cams, pose, steps, warmup, None, flush, clk_index)
    out = {"value": steps / t, "unit": "frames/s", "ms_per_step": 1e3 * t / steps,
           "stages_ms": {k: round(v, 5) for k, v in stages.items()},
           "workload": "same 2M anchors and 120-pose path; 10 explicit 3D Gaussians per anchor "
                       "(seeded attributes) in place of the decoders"}
    del rd
    torch.cuda.empty_cache()
    return out


def _appearance_bench(cams, pose, steps, warmup, flush, clk_index):
    """1080p frames/s of the BF16 neural form with per-anchor appearance codes (Sec. 4.4:
    an 8-value code per anchor in the colour decoder's first layer) on the same scene and path,
    without the gate: compare with the no-gate BF16 line."""
    import torch
    import synth
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, _ = _workload()
    sa, ma = synth.with_appearance(sc, mlp, seed=0)
    del sc
    W, H = cams[0].W, cams[0].H
    rd = Renderer(sa, ma, W, H, sel_cap=200_000, pair_cap=6_000_000, precision="bf16")
    rd.track_last = False
    for cam in cams:                      # size the buffers on every pose
        rd.render(cam)
    t, stages, clk = _time_form(rd, cams, pose, steps, warmup, None, flush, clk_index)
    out = {"value": steps / t, "unit": "frames/s", "ms_per_step": 1e3 * t / steps,
           "stages_ms": {k: round(v, 5) for k, v in stages.items()},
           "workload": f"same 2M anchors and 120-pose path; {sa.app.shape[1]}-value appearance "
                       "code per anchor (seeded N(0, 0.5)) fed to the colour decoder, BF16, "
                       "no gate"}
    del rd
    torch.cuda.empty_cache()
    return out


FIT_SIGMA = 0.05     # N(0, 0.05) added to the N(0, 0.1) anchor features after the targets


def _fit_targets(tr, cams, seed=1):
    """Targets the training steps can fit: every view rendered (training mode, untimed) from
    the scene as built, after which the anchor features get seeded N(0, FIT_SIGMA) noise, so
    the steps pull the perturbed scene back towards images it can produce.  (Against noise
    images, dense Adam at lr 1e-3 drives every decoded opacity below zero within two steps,
    after which no Gaussian is drawn and a step does almost no work.)  Returns the targets and
    the counts of every view before the perturbation (they also size the buffers)."""
    import torch
    targets, counts = [], []
    for cam in cams:
        c = tr.render(cam, infer=False)
        assert c.overflow == 0 and c.timeout == 0, "size the buffers for the target renders"
        targets.append(tr.img.clone())
        counts.append(c)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    tr.feat.add_(FIT_SIGMA * torch.randn(tr.feat.shape, generator=gen, device="cuda"))
    return targets, counts


def _pairs_kept(tr, cams, pairs0):
    """Pair count of the views after training over their count before it (untimed), so that a
    step time measured on a scene that stopped drawing shows: such a time is not valid."""
    now = [tr.render(cam, infer=False).n_pairs for cam in cams]
    return round(float(sum(now)) / max(1, sum(pairs0)), 4)


def _train_appearance_bench(clk_index, steps=60, warmup=5):
    """Training steps per second of the street workload (one 1600x900 view per step, L1,
    dense Adam) with an 8-value appearance code per anchor (Sec. 4.4), BF16: the codes and
    their weights are trained with everything else."""
    import torch
    import synth
    from paper_2403_17898_gb300.render import Trainer
    sc, mlp, cams = synth.CONFIGS["street500k_1600x900"]()
    sa, ma = synth.with_appearance(sc, mlp, seed=0)
    W, H = cams[0].W, cams[0].H
    tr = Trainer(sa, ma, W, H, sel_cap=400_000, pair_cap=8_000_000, precision="bf16")
    del sc, sa
    targets, cnt0 = _fit_targets(tr, cams)
    sel_max = max(c.n_selected for c in cnt0)
    pair_max = max(c.n_pairs for c in cnt0)
    tr.sel_cap, tr.pair_cap = int(sel_max * 1.2) + 1024, int(pair_max * 1.5) + 4096
    tr._alloc()
    batch = lambda i: ([cams[i % len(cams)]], [targets[i % len(cams)]])
    for i in range(warmup):
        tr.train_step(*batch(i))
    torch.cuda.synchronize()
    timers, ev = {}, []
    with ClockSampler(clk_index) as clk:
        for i in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            tr.train_step(*batch(warmup + i), timers=timers)
            e1.record()
            ev.append((e0, e1))
        torch.cuda.synchronize()
    c = tr.counts()
    assert c.overflow == 0 and c.timeout == 0, "overflow or expired wait in training"
    ms = [a.elapsed_time(b) for a, b in ev]
    kept = _pairs_kept(tr, cams, [c.n_pairs for c in cnt0])
    out = {"workload": "street500k_1600x900 with an 8-value appearance code per anchor "
                       "(codes and code weights trained), BF16, L1, dense Adam; targets: the "
                       "views rendered before N(0, 0.05) noise was added to the features",
           "pairs_kept": kept, "valid": kept > 0.5, "loss_last_step": float(tr.loss.item()),
           "train_steps_per_s": 1e3 * steps / float(np.sum(ms)),
           "ms_per_step": float(np.mean(ms)), "steps": steps, "warmup": warmup,
           "stages_ms_per_step": {k: round(float(np.sum([a.elapsed_time(b) for a, b in v]))
                                            / steps, 4) for k, v in timers.items()},
           "clocks": clk.summary()}
    del tr, targets
    torch.cuda.empty_cache()
    return out


def _train_bench(clk_index, steps_scale=1.0):
    """Training steps per second of both training workloads, plain FP32 decode and BF16
    decode: each step clears the gradients, runs forward + loss + backward for its views and
    one Adam update (device time, CUDA events around every step)."""
    import torch
    import synth
    from paper_2403_17898_gb300.render import Trainer
    out = {}
    for name, vps, lam, K, Wm, desc in TRAIN_WORKLOADS:
        K = max(2, int(round(K * steps_scale)))
        sc, mlp, cams = synth.CONFIGS[name]()
        W, H = cams[0].W, cams[0].H
        stride = max(1, len(cams) // 16) if vps > 1 else 1
        views = cams[::stride][:vps] if vps > 1 else cams
        tr = Trainer(sc, mlp, W, H, ssim_lambda=lam, sel_cap=400_000, pair_cap=8_000_000,
                     track_view_frequency=True, track_growth=True, track_opacity=True)
        voxel = synth.voxel_sizes(sc)
        del sc
        n_t = len(views)
        # the targets (views rendered before the features are perturbed) also size the
        # buffers, with headroom for the updates
        targets, cnt0 = _fit_targets(tr, views)
        sel_max = max(c.n_selected for c in cnt0)
        pair_max = max(c.n_pairs for c in cnt0)
        tr.sel_cap, tr.pair_cap = int(sel_max * 1.2) + 1024, int(pair_max * 1.5) + 4096
        tr._alloc()
        res = {"workload": desc, "anchors": int(tr.N), "views_per_step": vps,
               "resolution": f"{W}x{H}", "ssim_lambda": lam, "steps": K, "warmup": Wm,
               "l2": "no flush: every step streams the dense Adam state (>= 1 GB) through L2",
               "pipelined_views": "each view's loss and backward run on a second stream while "
                                  "the next view's forward runs (two sets of per-view buffers), "
                                  "so the per-stage times of a step overlap and add up to more "
                                  "than the step",
               "max_selected": sel_max, "max_pairs": pair_max}
        # both forms start from the same parameters and optimiser state
        init = {n: t.clone() for n, t in tr._anchor_params().items()}
        init.update({"mlp." + n: t.clone() for n, t in tr.mlp.items()})
        for precision in ("fp32", "bf16"):
            for n, t in tr._anchor_params().items():
                t.copy_(init[n])
            for n, t in tr.mlp.items():
                t.copy_(init["mlp." + n])
            for t in list(tr.adam_m.values()) + list(tr.adam_v.values()):
                t.zero_()
            tr.zero_grad()
            tr.step_count = 0
            tr.sel_count.zero_()
            tr.n_views_seen = 0
            tr.precision = precision
            batch = lambda i: ([views[(i * vps + v) % len(views)] for v in range(vps)],
                               [targets[(i * vps + v) % n_t] for v in range(vps)])
            for i in range(Wm):
                tr.train_step(*batch(i))
                if i == 0:
                    loss_first = float(tr.loss.item())
            torch.cuda.synchronize()
            timers, ev = {}, []
            with ClockSampler(clk_index) as clk:
                for i in range(K):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    tr.train_step(*batch(Wm + i), timers=timers)
                    e1.record()
                    ev.append((e0, e1))
                torch.cuda.synchronize()
            c = tr.counts()
            assert c.overflow == 0 and c.timeout == 0, "overflow or expired wait in training"
            ms = [a.elapsed_time(b) for a, b in ev]
            stages = {k: round(float(np.sum([a.elapsed_time(b) for a, b in v])) / K, 4)
                      for k, v in timers.items()}
            loss_last = float(tr.loss.item())
            kept = _pairs_kept(tr, views, [c.n_pairs for c in cnt0])
            if precision == "bf16":
                # view-frequency pruning (Sec. 4.2.2) after the counted training views
                n_before, n_views = tr.N, tr.n_views_seen
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                n_after = tr.prune(PRUNE_TAU_V)
                torch.cuda.synchronize()
                res["view_frequency_prune"] = {
                    "tau_v": PRUNE_TAU_V, "views_counted": n_views, "anchors_before": n_before,
                    "anchors_after": n_after, "seconds": time.perf_counter() - t0,
                    "note": "count, order-preserving compaction and gather of every per-anchor "
                            "array and its Adam state, all on the GPU"}
                # average-opacity pruning (Sec. 4.2.2) from the same views' statistic
                n_before = tr.N
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                n_after = tr.prune_opacity(PRUNE_TAU_O)
                torch.cuda.synchronize()
                res["opacity_prune"] = {
                    "tau_o": PRUNE_TAU_O, "anchors_before": n_before, "anchors_after": n_after,
                    "seconds": time.perf_counter() - t0,
                    "note": "average opacity of each anchor's Gaussians over the counted views; "
                            "anchors below tau_o removed with the same compaction"}
                # next-level growing + LOD-bias update (Sec. 4.2.1) from the statistics of the
                # same training views (accumulated inside every timed step)
                seen = int((tr.grad_cnt > 0).sum().item())
                n_before = tr.N
                dL0 = tr.dL.clone()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                added = tr.grow(voxel, tau_g=GROW_TAU_G, beta=GROW_BETA, eps=GROW_EPS)
                torch.cuda.synchronize()
                res["anchor_growth"] = {
                    "tau_g": GROW_TAU_G, "beta": GROW_BETA, "eps": GROW_EPS,
                    "gaussians_with_statistics": seen, "anchors_before": n_before,
                    "anchors_added": added,
                    "lod_bias_raised": int((tr.dL[:n_before] != dL0).sum().item()),
                    "seconds": time.perf_counter() - t0,
                    "note": "LOD-bias update, voxel-hash proposals, first-proposal-wins "
                            "compaction, appended rows with the parents' features and fresh "
                            "Adam state, all on the GPU (a few steps from a perturbed scene: "
                            "the statistics are not those of a converged one)"}
            res[precision] = {"train_steps_per_s": 1e3 * K / float(np.sum(ms)),
                              "ms_per_step": float(np.mean(ms)), "stages_ms_per_step": stages,
                              "loss_first_step": loss_first, "loss_last_step": loss_last,
                              "pairs_kept": kept, "valid": kept > 0.5,
                              "clocks": clk.summary()}
        out[name] = res
        del tr, targets
        torch.cuda.empty_cache()
    return out


POS_WEIGHT = 4.0


def _train_proposal(rd, train_cams, test_cams, full_rd):
    """Trains the anchor-visibility proposal on the training poses (BCE with positives
    weighted, so dropping a visible anchor costs more than keeping an invisible one),
    calibrates p* on every 5th training pose as the largest threshold whose pooled PSNR loss
    stays within the budget, and assesses it on the held-out poses against full-detail renders
    (pooled and per view).  If the held-out poses exceed the budget, the plain LOD path is used
    (the gate's fallback)."""
    import synth
    from paper_2403_17898_gb300 import proposal
    t0 = time.perf_counter()
    views = proposal.collect_labels(rd, train_cams)
    net = proposal.ProposalNet(synth.proposal_mlp(seed=0), lr=2e-3)
    hist = proposal.train(net, rd, views, epochs=30, pos_weight=POS_WEIGHT)
    t_train = time.perf_counter() - t0

    calib = train_cams[::5]
    p_star, curve = proposal.calibrate(rd, full_rd, calib, net.w, DPSNR_GATE_DB)
    held = proposal.assess(rd, full_rd, test_cams, (net.w, p_star)) if p_star > 0 else None
    pooled = held.pooled_db if held is not None else 0.0
    use_gate = p_star > 0 and pooled <= DPSNR_GATE_DB
    per_view = None
    if held is not None:
        d = held.dpsnr
        worst = int(np.argmax(d))
        per_view = {
            "psnr_plain_db": [round(x, 3) for x in held.psnr_plain],
            "psnr_gated_db": [round(x, 3) for x in held.psnr_gated],
            "kept_frac": [round(x, 4) for x in held.kept],
            "worst_view": {"index": worst, "psnr_plain_db": held.psnr_plain[worst],
                           "psnr_gated_db": held.psnr_gated[worst], "dpsnr_db": d[worst]},
            "psnr_plain_db_min": float(np.min(held.psnr_plain)),
            "psnr_gated_db_min": float(np.min(held.psnr_gated))}
    med = float(np.median(held.dpsnr)) if held is not None else 0.0
    mx = float(np.max(held.dpsnr)) if held is not None else 0.0
    kept = float(np.mean(held.kept)) if held is not None else 1.0
    curve = [[round(x, 4) for x in row] for row in curve]
    info = {"train_poses": len(train_cams), "heldout_poses": len(test_cams),
            "epochs": len(hist), "bce_first_epoch": hist[0], "bce_last_epoch": hist[-1],
            "pos_weight": POS_WEIGHT, "train_s": t_train, "p_star": p_star,
            "label": "max T*alpha >= 1/255",
            "calibration_curve[p*, dPSNR set, dPSNR view median, dPSNR view max, kept]": curve,
            "heldout_dpsnr_db_set": pooled, "heldout_dpsnr_db_view_median": med,
            "heldout_dpsnr_db_view_max": mx, "heldout_kept_anchor_frac": kept,
            "heldout_per_view": per_view,
            "p_star_calibrated_on": f"{len(calib)} of the training poses (every 5th)",
            "gate_used": use_gate,
            "dpsnr_definition": "10 log10(sum_v MSE(gated BF16_v, full_v) / sum_v MSE(plain FP32_v, "
                                "full_v)) over the views: the PSNR of the view set, full = "
                                "every level selected; per-view PSNR differences beside it"}
    return net, p_star, use_gate, info


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import synth
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2403_17898_gb300 import build as _b
    _b.build()
    from paper_2403_17898_gb300.render import Renderer

    sc, mlp, cams = _workload()
    n = len(cams)
    W, H = cams[0].W, cams[0].H
    rd = Renderer(sc, mlp, W, H, sel_cap=200_000, pair_cap=4_000_000)
    pose = pose_of(rank, ws, n)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 126 MB L2

    # the learned proposal (trained on its own poses of the same scene, assessed on held-out)
    train_cams = synth.proposal_poses(cams, 200, seed=2)
    test_cams = synth.proposal_poses(cams, 60, seed=3)
    full_rd = Renderer(sc, mlp, W, H, sel_cap=2_000_000, pair_cap=40_000_000)
    net, p_star, use_gate, pinfo = _train_proposal(rd, train_cams, test_cams, full_rd)
    del full_rd
    torch.cuda.empty_cache()
    gate = (net.w, p_star) if use_gate else None
    # inference frames: no backward follows, so the blend does not record each pixel's last
    # blended entry (image and T are bit-identical either way)
    rd.track_last = False

    # plain FP32 form
    rd.precision = "fp32"
    work_plain = _per_pose(rd, cams)
    if ws > 1:
        dist.barrier()
    t_plain, stages_plain, _ = _time_form(rd, cams, pose, args.steps, args.warmup, None, flush,
                                          local)
    # BF16 decode alone (what the gate is compared with)
    rd.precision = "bf16"
    t_bf16, stages_bf16, _ = _time_form(rd, cams, pose, args.steps, args.warmup, None, flush,
                                        local)
    # BF16 decode + learned gate: the measured form
    work = _per_pose(rd, cams, gate)
    if ws > 1:
        dist.barrier()
    total_s, mean_ms, clocks = _time_form(rd, cams, pose, args.steps, args.warmup, gate, flush,
                                          local)
    if ws > 1:
        dist.barrier()
    t_max, tp_max, tb_max = max_over_ranks([total_s, t_plain, t_bf16], ws, "cuda")
    fps = ws * args.steps / t_max
    fps_plain = ws * args.steps / tp_max
    fps_bf16 = ws * args.steps / tb_max

    # end-to-end through the public calls: every view's image lands in pinned host memory.
    # The sequence call copies view i to the host while view i + 1 renders; the single-view
    # call (the blend writes straight into pinned host memory, then wait) and the sequence
    # call in that zero-copy form are reported beside it.
    hosts = [torch.empty(3, H, W, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    n_e2e = min(args.steps, 600)
    e2e_cams = [cams[pose(i)] for i in range(n_e2e)]
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    rd.render_sequence_to_host(e2e_cams, hosts, gate=gate)
    e2e_s = max_over_ranks([time.perf_counter() - t0], ws, "cuda")[0]
    e2e_fps = ws * n_e2e / e2e_s
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for cam in e2e_cams:
        rd.render_to_host(cam, hosts[0], gate=gate)
    e2e_sync_s = max_over_ranks([time.perf_counter() - t0], ws, "cuda")[0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rd.render_sequence_to_host(e2e_cams, hosts, gate=gate, zero_copy=True)
    e2e_zc_s = max_over_ranks([time.perf_counter() - t0], ws, "cuda")[0]

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0

    peaks, src = _peaks()
    timed = [pose(args.warmup + i) for i in range(args.steps)]
    dominant = max(mean_ms, key=mean_ms.get)
    evals = float(np.mean([work[p][3] for p in timed]))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = SM_COUNT * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12          # Tops/s
    stages = {}
    for k, v in mean_ms.items():
        if k == "proposal_gate":
            continue
        b = float(np.mean([stage_bytes(sc.N, work[p][0], work[p][1], work[p][2],
                                       rd.gx * rd.gy, W * H)[k] for p in timed]))
        stages[k] = {"ms": v, "algorithmic_GB_per_s": b / (v * 1e-3) / 1e9,
                     "hbm_frac": b / (v * 1e-3) / 1e9 / peaks["hbm_gbs"]}
    if dominant == "blend_fwd":
        ach = evals * OPS_PER_EVAL / (mean_ms["blend_fwd"] * 1e-3) / 1e12
        roof = {"kernel": "blend_fwd", "bound": "alu", "achieved": ach, "peak": alu_peak,
                "unit": "TFLOP/s", "frac": ach / alu_peak, "traffic": BLEND_FWD_DRAM_BYTES,
                "traffic_note": BLEND_FWD_TRAFFIC_NOTE,
                "issue_active_frac_ncu": BLEND_FWD_ISSUE_FRAC,
                "work": f"{evals:.4g} (pixel, Gaussian) tests executed per frame (n_eval: the "
                        f"entries of each pixel's warp-block list up to its stop) x "
                        f"{OPS_PER_EVAL} FP32 ops",
                "peak_source": f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                               f"{sm_max:.0f} MHz ({src} sm_max_mhz)"}
    else:
        gbs = stages[dominant]["algorithmic_GB_per_s"]
        roof = {"kernel": dominant, "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                "peak_source": f"{src} hbm_gbs"}
    mean = lambda w, i: float(np.mean([w[p][i] for p in timed]))
    line = {
        "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 decode GEMMs, f32 accumulate/blend",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC.replace(
                       "FP32 decode", "BF16 decode + learned gate" if use_gate else
                       "BF16 decode (learned gate fell back to the plain LOD path)"),
                   "anchors": sc.N, "levels": sc.NL, "resolution": f"{W}x{H}", "poses": n,
                   "parallelism": f"replicas x{ws}",
                   "l2": "256 MB buffer written between timed steps (L2 is 126 MB)",
                   "mean_selected_anchors": mean(work, 0), "mean_gaussians": mean(work, 1),
                   "mean_pairs": mean(work, 2), "mean_evaluations": evals},
        "plain_fp32": {"value": fps_plain, "unit": "frames/s",
                       "ms_per_step": 1e3 * t_plain / args.steps,
                       "stages_ms": {k: round(v, 5) for k, v in stages_plain.items()},
                       "mean_selected_anchors": mean(work_plain, 0),
                       "mean_pairs": mean(work_plain, 2),
                       "mean_evaluations": mean(work_plain, 3)},
        "bf16_no_gate": {"value": fps_bf16, "unit": "frames/s",
                         "ms_per_step": 1e3 * t_bf16 / args.steps,
                         "stages_ms": {k: round(v, 5) for k, v in stages_bf16.items()}},
        "speedup_vs_plain_fp32": fps / fps_plain,
        "gate_speedup_vs_bf16_no_gate": fps / fps_bf16,
        "proposal": pinfo,
        "roofline": roof,
        "stages_ms": {k: round(v, 5) for k, v in mean_ms.items()},
        "stages": stages,
        "clocks": clocks,
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": 88,
                "d2h_bytes_per_step": 3 * W * H * 4, "steps": n_e2e,
                "call": "Renderer.render_sequence_to_host (every view rendered and its image "
                        "copied to pinned host memory; the copy of view i overlaps the "
                        "rendering of view i + 1)",
                "single_view_call": {"value": ws * n_e2e / e2e_sync_s, "unit": "frames/s",
                                     "call": "Renderer.render_to_host per view (the blend "
                                             "writes the image into pinned host memory, "
                                             "wait)"},
                "zero_copy_sequence_call": {"value": ws * n_e2e / e2e_zc_s,
                                            "unit": "frames/s",
                                            "call": "render_sequence_to_host(zero_copy=True):"
                                                    " every blend writes into pinned host "
                                                    "memory, one view in flight"}},
        "gpu_launches": args.steps * (LAUNCHES["lod_select_gated" if use_gate else "lod_select"]
                                      + LAUNCHES["decode_project"] + LAUNCHES["sort"]
                                      + LAUNCHES["blend_fwd"]),
    }
    def extra(fn, *a):
        """An additional measurement; a failure is recorded in the line instead of losing it."""
        try:
            return fn(*a)
        except Exception as e:                       # noqa: BLE001 - reported, not hidden
            return {"error": f"{type(e).__name__}: {e}"[:300]}

    if ws == 1 and not args.no_train:
        del rd
        torch.cuda.empty_cache()
        line["explicit_3dgs"] = extra(_explicit_bench, cams, pose, min(args.steps, 600),
                                      args.warmup, flush, local)
        line["appearance_codes"] = extra(_appearance_bench, cams, pose, min(args.steps, 600),
                                         args.warmup, flush, local)
        line["train"] = extra(_train_bench, local)
        if "error" not in line["train"]:
            line["train"]["street500k_1600x900_appearance"] = extra(_train_appearance_bench,
                                                                    local)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(*_as_f64(sc, mlp), cams)
        line["cpu_baseline"]["single_thread"] = extra(cpu_baseline_single_thread)
        if not args.no_train:
            line["cpu_baseline"]["train_step_city8M"] = extra(cpu_baseline_train_view)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_profile(args):
    """Renders warmup + steps frames of the workload (BF16 decode, no gate) and exits: the
    small case that the ncu captures under profiles/ are taken on."""
    import torch
    from paper_2403_17898_gb300 import build as _b
    _b.build()
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cams = _workload()
    rd = Renderer(sc, mlp, cams[0].W, cams[0].H, sel_cap=200_000, pair_cap=4_000_000,
                  precision=args.precision)
    rd.track_last = False            # as the timed inference frames
    gate = None
    if args.gate:
        # an untrained proposal network at p* = 0.5: the gate kernel's cost, not its quality
        import synth
        from paper_2403_17898_gb300 import proposal
        gate = (proposal.ProposalNet(synth.proposal_mlp(seed=0)).w, 0.5)
    for i in range(args.warmup + args.steps):
        rd.render(cams[(37 * i + 60) % len(cams)], gate=gate)
    torch.cuda.synchronize()
    print(json.dumps({"profile_frames": args.warmup + args.steps, **rd.counts().__dict__}))
    return 0


def run_profile_train(args):
    """A few training steps (L1 + D-SSIM): by default one 1600x900 view of the 500k-anchor
    street workload per step (the small case the training-kernel ncu captures are taken on),
    or the 16-view steps of the 8M-anchor city (for a launch list)."""
    import torch
    import synth
    from paper_2403_17898_gb300 import build as _b
    _b.build()
    from paper_2403_17898_gb300.render import Trainer
    sc, mlp, cams = synth.CONFIGS[args.train_workload]()
    W, H = cams[0].W, cams[0].H
    tr = Trainer(sc, mlp, W, H, ssim_lambda=0.2, sel_cap=100_000, pair_cap=2_000_000,
                 precision=args.precision, track_view_frequency=True, track_growth=True,
                 track_opacity=True)
    views = cams[::4][:16] if args.train_workload == "city8M_1080p" else [cams[len(cams) // 2]]
    tgts, cnt0 = _fit_targets(tr, views)
    for _ in range(args.warmup + args.steps):
        tr.train_step(views, tgts)
    torch.cuda.synchronize()
    c = tr.counts()
    assert c.overflow == 0 and c.timeout == 0
    print(json.dumps({"profile_train_steps": args.warmup + args.steps,
                      "pairs_kept": _pairs_kept(tr, views, [c.n_pairs for c in cnt0]),
                      **c.__dict__}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-train", action="store_true",
                    help="skip the training-step measurements")
    ap.add_argument("--profile", action="store_true",
                    help="render a few frames only (the case profiled with ncu)")
    ap.add_argument("--gate", action="store_true",
                    help="with --profile: also run the proposal gate (untrained network)")
    ap.add_argument("--profile-train", action="store_true",
                    help="run a few training steps only (the case training kernels are profiled on)")
    ap.add_argument("--train-workload", default="street500k_1600x900",
                    choices=["street500k_1600x900", "city8M_1080p"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--cpu-single", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_single:
        return run_cpu_single(args)
    if args.profile:
        return run_profile(args)
    if args.profile_train:
        return run_profile_train(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
