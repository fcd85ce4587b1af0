"""Anchor growing and the LOD-bias update (Sec. 4.2.1) through the CUDA path, against the
oracle on seeded synthetic statistics.

The decisions (threshold tests, the voxel a Gaussian falls in, the first proposal of a shared
voxel) are taken in FP32 with the same rounded steps on both sides, so the new anchors, their
order and their parents are compared bit for bit, on the 4k-anchor cube (loop oracle) and on
the 2M-anchor city (array oracle).  The per-view statistics are compared within FP32
summation error.  The Trainer's densification step is checked end to end: rows appended
with their parents' features, a frame equal to a fresh renderer's, training continuing."""
import copy

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import cuda, lib_ready

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    return lib_ready()


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _stats(N, k, seed, tau0, seen=0.6):
    """Seeded statistics: a view count 0..5 per Gaussian (zero for a 1 - seen fraction) and
    summed norms whose averages spread log-normally around tau0."""
    rng = np.random.default_rng(seed)
    cnt = rng.integers(1, 6, size=(N, k)) * (rng.uniform(size=(N, k)) < seen)
    avg = rng.lognormal(np.log(tau0), 0.7, size=(N, k))
    return (avg * cnt).astype(np.float32), cnt.astype(np.int64)


def _voxels(sc):
    return synth.voxel_sizes(sc)


def _gpu_grow(abi, torch, sc, acc, cnt, tau, vox, max_new, next_level=True):
    N, k = acc.shape
    scr = torch.empty(abi.grow_scratch_bytes(N, k), dtype=torch.uint8, device="cuda")
    cap = max(max_new, 1)
    out = (torch.full((cap, 3), -1.0, device="cuda"),
           torch.full((cap,), 99, dtype=torch.uint8, device="cuda"),
           torch.full((cap, 3), -1.0, device="cuda"),
           torch.full((cap,), -1, dtype=torch.int32, device="cuda"))
    n_new = torch.full((2,), 7, dtype=torch.int32, device="cuda")
    abi.grow_anchors(cuda(sc.pos), cuda(sc.level), cuda(sc.offs), cuda(sc.lv), cuda(acc),
                     cuda(cnt.astype(np.int32)), N, k, sc.NL, tau, vox, *out, max_new, n_new, scr,
                     next_level=next_level)
    torch.cuda.synchronize()
    n, need = (int(x) for x in n_new.cpu().numpy().view(np.uint32))
    p, L, s, par = (t.cpu().numpy() for t in out)
    return n, need, p[:n], L[:n], s[:n], par[:n].astype(np.int64)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_grow_matches_oracle_cube(abi, torch, seed):
    sc, _, _ = synth.CONFIGS["cube4k_128"]()
    tau, _ = oracle.grow_thresholds(2e-4, 0.2, sc.NL)
    vox = _voxels(sc)
    acc, cnt = _stats(sc.N, sc.k, seed, tau[1])
    ref = oracle.grow_anchors(sc.pos, sc.level, sc.offs, sc.lv, acc, cnt, sc.NL, tau, vox)
    n, need, *got = _gpu_grow(abi, torch, sc, acc, cnt, tau, vox, sc.N * sc.k)
    print(f"cube seed {seed}: {need} new anchors, levels {np.bincount(ref[1], minlength=sc.NL)}")
    assert n == need == len(ref[0]) > 100
    assert len(np.unique(ref[1])) >= 2
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    # a smaller output buffer: the first rows, and the size needed
    m = need // 3
    n2, need2, *part = _gpu_grow(abi, torch, sc, acc, cnt, tau, vox, m)
    assert n2 == m and need2 == need
    for a, b in zip(part, ref):
        assert np.array_equal(a, b[:m])


def test_grow_edge_cases(abi, torch):
    sc, _, _ = synth.CONFIGS["cube4k_128"]()
    tau, _ = oracle.grow_thresholds(2e-4, 0.2, sc.NL)
    vox = _voxels(sc)
    # nothing seen: nothing grows
    acc = np.zeros((sc.N, sc.k), np.float32)
    cnt = np.zeros((sc.N, sc.k), np.int64)
    assert _gpu_grow(abi, torch, sc, acc, cnt, tau, vox, 100)[:2] == (0, 0)
    # every Gaussian far above every threshold: all proposals at the next level (or the finest)
    acc[:], cnt[:] = 1.0, 1
    ref = oracle.grow_anchors(sc.pos, sc.level, sc.offs, sc.lv, acc, cnt, sc.NL, tau, vox)
    n, need, *got = _gpu_grow(abi, torch, sc, acc, cnt, tau, vox, sc.N * sc.k)
    assert n == len(ref[0])
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    assert (got[1] >= 1).all()
    # an empty anchor set
    empty = copy.copy(sc)
    for name in ("pos", "level", "offs", "lv"):
        setattr(empty, name, getattr(sc, name)[:0])
    res = _gpu_grow(abi, torch, empty, np.zeros((0, sc.k), np.float32),
                    np.zeros((0, sc.k), np.int64), tau, vox, 10)
    assert res[:2] == (0, 0)


def test_grow_matches_oracle_city(abi, torch):
    """2M anchors x 10 Gaussians: a hash table of 2^26 slots, ~10^5 proposals."""
    sc, _, _ = synth.CONFIGS["city2M_1080p"]()
    tau, _ = oracle.grow_thresholds(2e-4, 0.2, sc.NL)
    vox = _voxels(sc)
    acc, cnt = _stats(sc.N, sc.k, 7, tau[2], seen=0.05)
    ref = oracle.grow_anchors_vectorized(sc.pos, sc.level, sc.offs, sc.lv, acc, cnt, sc.NL,
                                         tau, vox)
    n, need, *got = _gpu_grow(abi, torch, sc, acc, cnt, tau, vox, len(ref[0]) + 10)
    print(f"city: {need} new anchors of {sc.N}, levels {np.bincount(ref[1], minlength=sc.NL)}")
    assert n == need == len(ref[0]) > 10_000
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_accumulate_matches_oracle(abi, torch):
    rng = np.random.default_rng(3)
    N, k, M, W, H = 5000, 10, 1777, 320, 200
    acc_ref = cnt_ref = None
    acc = torch.zeros(N, k, device="cuda")
    cnt = torch.zeros(N, k, dtype=torch.int32, device="cuda")
    for view in range(3):
        sel = np.sort(rng.choice(N, size=M, replace=False))
        G = M * k
        drec = rng.normal(0, 1e-5, size=(G, 9)).astype(np.float32)
        tiles = (rng.uniform(size=G) < 0.7) * rng.integers(1, 9, size=G)
        counts = np.zeros(8, np.uint32)
        counts[0], counts[1] = M, G
        abi.grow_accumulate(cuda(drec), cuda(tiles.astype(np.int32)), cuda(sel.astype(np.int32)),
                            cuda(counts.view(np.int32)), k, W, H, acc, cnt)
        acc_ref, cnt_ref = oracle.grow_accumulate(N, k, sel, drec, tiles, W, H, acc_ref, cnt_ref)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cnt.cpu().numpy(), cnt_ref)
    np.testing.assert_allclose(acc.cpu().numpy(), acc_ref, rtol=1e-6, atol=1e-12)


def test_lod_bias_update_matches_oracle(abi, torch):
    sc, _, _ = synth.CONFIGS["cube4k_128"]()
    _, bias = oracle.grow_thresholds(2e-4, 0.2, sc.NL)
    acc, cnt = _stats(sc.N, sc.k, 4, bias[1])
    rng = np.random.default_rng(4)
    dL = rng.normal(0, 0.3, sc.N).astype(np.float32)
    ref = oracle.lod_bias_update(sc.level, acc, cnt, bias, 0.01, dL)
    d = cuda(dL)
    abi.update_lod_bias(cuda(sc.level), cuda(acc), cuda(cnt.astype(np.int32)), sc.N, sc.k,
                        sc.NL, bias, 0.01, d)
    torch.cuda.synchronize()
    got = d.cpu().numpy()
    assert np.array_equal(got, ref)
    assert 0 < np.count_nonzero(got != dL) < sc.N


def test_trainer_grows_and_keeps_training(abi, torch):
    from paper_2403_17898_gb300.render import Renderer, Trainer
    sc, mlp, _ = synth.CONFIGS["cube4k_128"]()
    sa, ma = synth.with_appearance(sc, mlp, seed=2)
    rng = np.random.default_rng(5)
    views = [synth.look_at_camera(rng.uniform(-15, 15, 3) + np.array([0, 0, 12.0]),
                                  rng.uniform(-2, 2, 3), 128, 128, d_max=30.0) for _ in range(4)]
    tr = Trainer(sa, ma, 128, 128, track_growth=True, track_view_frequency=True,
                 sel_cap=sc.N * 2, pair_cap=1 << 21)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    tgts = [torch.rand(3, 128, 128, generator=gen, device="cuda") for _ in views]
    tr.train_step(views, tgts)
    tr.train_step(views, tgts)
    cnt = tr.grad_cnt.cpu().numpy()
    assert cnt.max() <= 2 * len(views) and cnt.sum() > 0
    assert (tr.grad_acc.cpu().numpy() >= 0).all()
    N0 = tr.N
    feat0 = tr.feat.clone()
    dL0 = tr.dL.cpu().numpy()
    # thresholds scaled to the synthetic gradients so that some anchors grow
    avg = tr.grad_acc.cpu().numpy()[cnt > 0] / cnt[cnt > 0]
    tau_g = float(np.quantile(avg, 0.98))
    n = tr.grow(_voxels(sc), tau_g=tau_g, beta=0.2, eps=0.01)
    assert n > 0 and tr.N == N0 + n
    dd = tr.dL.cpu().numpy()[:N0] - dL0
    assert np.all((dd == 0) | (np.abs(dd - 0.01) < 1e-6)) and (dd != 0).any()
    assert not tr.dL[N0:].any() and not tr.offs[N0:].any()
    assert torch.equal(tr.feat[:N0], feat0)
    for name in ("feat", "offs", "lv", "app"):
        assert tr.adam_m[name].shape[0] == tr.N and not tr.adam_m[name][N0:].any()
    assert tr.grad_acc.shape[0] == tr.N and not tr.grad_acc.any()
    # each new anchor carries its parent's features: every new feature row is an old row
    old = {r.tobytes() for r in feat0.cpu().numpy()}
    assert all(r.tobytes() in old for r in tr.feat[N0:].cpu().numpy())
    # the grown set renders like a fresh renderer of the same arrays, and keeps training
    sp = copy.copy(sa)
    for name in ("pos", "level", "dL", "feat", "offs", "lv", "app"):
        setattr(sp, name, getattr(tr, name).cpu().numpy())
    mp = copy.copy(ma)
    for name in ("w1", "b1", "w2_op", "b2_op", "w2_col", "b2_col", "w2_cov", "b2_cov", "w1_app"):
        setattr(mp, name, tr.mlp[name].cpu().numpy())
    fresh = Renderer(sp, mp, 128, 128)
    for v in views[:2]:
        tr.render(v)
        fresh.render(v)
        assert torch.equal(tr.img, fresh.img)
    tr.train_step(views, tgts)
    c = tr.counts()
    assert c.overflow == 0 and c.timeout == 0
    assert tr.grad_cnt.sum().item() > 0


def test_grow_without_next_level_matches_oracle(abi, torch):
    """The progressive stage (Sec. 4.3) grows at the Gaussian's own level only."""
    sc, _, _ = synth.CONFIGS["cube4k_128"]()
    tau, _ = oracle.grow_thresholds(2e-4, 0.2, sc.NL)
    vox = _voxels(sc)
    acc, cnt = _stats(sc.N, sc.k, 8, tau[1])
    ref = oracle.grow_anchors(sc.pos, sc.level, sc.offs, sc.lv, acc, cnt, sc.NL, tau, vox,
                              next_level=False)
    n, need, *got = _gpu_grow(abi, torch, sc, acc, cnt, tau, vox, sc.N * sc.k, next_level=False)
    assert n == need == len(ref[0]) > 100
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_progressive_training_caps_the_levels(abi, torch):
    """Progressive training (Sec. 4.3): the Trainer's schedule matches the oracle's, each
    step selects only anchors up to the active level (the selection of a capped tree equals
    the oracle's selection on that tree), and growing has no next-level promotion while the
    stage lasts."""
    from paper_2403_17898_gb300.render import Trainer, progressive_schedule
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    assert progressive_schedule(8, 10_000, 1.5) == oracle.progressive_schedule(8, 10_000, 1.5)
    cam = cams[0]
    tr = Trainer(sc, mlp, 128, 128, progressive=(4, 1.5), track_growth=True)
    st = oracle.progressive_schedule(sc.NL, 4, 1.5)
    tgt = [torch.rand(3, 128, 128, device="cuda")]
    seen = []
    for it in range(6):
        L = tr.active_level()
        assert L == (oracle.active_level(st, it) if it < 4 else sc.NL - 1)
        assert tr.in_progressive_stage() == (it < 4)
        tr.train_step([cam], tgt)
        sel = tr.sel_idx[:tr.counts().n_selected].cpu().numpy()
        assert sc.level[sel].max() <= L
        # the same kept set as the oracle's selection on a tree of L + 1 levels, away from
        # knife-edge decisions
        idx, _, margin = oracle.lod_select(sc.pos, sc.level, sc.dL, L + 1, cam, False)
        sure = margin >= 1e-4
        ref = np.zeros(sc.N, bool)
        ref[idx] = True
        mine = np.zeros(sc.N, bool)
        mine[sel] = True
        assert np.array_equal(ref[sure], mine[sure])
        seen.append(L)
    assert seen[0] == sc.NL // 2 and seen[-1] == sc.NL - 1
