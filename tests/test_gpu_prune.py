"""GPU parity of view-frequency pruning (Sec. 4.2.2): per-anchor selection counts over
several views, the order-preserving list of kept anchors, the row gather that compacts the
anchor arrays, and a Trainer that prunes after counting its training views."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import SEL_MARGIN, cuda, lib_ready, to_np_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    return lib_ready()


def _views(n, seed):
    rng = np.random.default_rng(seed)
    return [synth.look_at_camera(rng.uniform(-15, 15, 3) + np.array([0, 0, 12.0]),
                                 rng.uniform(-2, 2, 3), 128, 128, d_max=30.0) for _ in range(n)]


def test_counts_over_views_match_oracle(abi):
    import torch
    sc, mlp, _ = synth.CONFIGS["cube4k_128"]()
    views = _views(7, 1)
    sels, knife = [], set()
    for v in views:
        idx, _, margin = oracle.lod_select(sc.pos, sc.level, sc.dL, sc.NL, v, False)
        sels.append(idx)
        knife |= set(np.nonzero(margin < SEL_MARGIN)[0].tolist())
    ref = oracle.view_frequency_counts(sc.N, sels)
    sel_count = torch.zeros(sc.N, dtype=torch.int32, device="cuda")
    cap = sc.N
    sel = torch.zeros(cap, dtype=torch.int32, device="cuda")
    w = torch.zeros(cap, device="cuda")
    counts = torch.zeros(8, dtype=torch.int32, device="cuda")
    scr = torch.empty(abi.lod_select_scratch_bytes(sc.N), dtype=torch.uint8, device="cuda")
    for v in views:
        counts.zero_()
        abi.lod_select(cuda(sc.pos), cuda(sc.level), cuda(sc.dL), sc.N, sc.NL, sc.k, v, False,
                       sel, w, cap, counts, scr)
        abi.count_selected(sel, counts, sel_count)
    torch.cuda.synchronize()
    got = sel_count.cpu().numpy().astype(np.int64)
    sure = np.setdiff1d(np.arange(sc.N), np.array(sorted(knife), np.int64))
    assert np.array_equal(got[sure], ref[sure])


@pytest.mark.parametrize("N", [1, 2047, 2048, 300_001])
def test_prune_list_matches_oracle(abi, N):
    import torch
    rng = np.random.default_rng(N)
    n_views = 37
    count = rng.integers(0, n_views + 1, size=N).astype(np.int64)
    count[rng.uniform(size=N) < 0.3] = 0
    for tau in (0.0, 0.01, 0.2, 0.7, 1.0):
        ref = oracle.prune_by_view_frequency(count, n_views, tau)
        keep = torch.full((N,), -1, dtype=torch.int32, device="cuda")
        n_kept = torch.zeros(1, dtype=torch.int32, device="cuda")
        scr = torch.empty(abi.prune_scratch_bytes(N), dtype=torch.uint8, device="cuda")
        abi.prune_anchors(cuda(count.astype(np.int32)), N, oracle.min_count_for(n_views, tau),
                          keep, n_kept, scr)
        torch.cuda.synchronize()
        n = int(n_kept.item())
        assert n == len(ref)
        assert np.array_equal(to_np_u32(keep)[:n].astype(np.int64), ref)


def test_gather_rows_matches_indexing(abi):
    import torch
    rng = np.random.default_rng(2)
    N, n = 5000, 1234
    idx = np.sort(rng.choice(N, n, replace=False)).astype(np.int32)
    f = rng.normal(size=(N, 10, 3)).astype(np.float32)
    b = rng.integers(0, 255, size=N).astype(np.uint8)
    nd = cuda(np.array([n], np.int32))
    fo = torch.zeros(n, 10, 3, device="cuda")
    bo = torch.zeros(n, dtype=torch.uint8, device="cuda")
    abi.gather_rows(cuda(f), fo, 120, cuda(idx), nd, n)
    abi.gather_rows(cuda(b), bo, 1, cuda(idx), nd, n)
    torch.cuda.synchronize()
    assert np.array_equal(fo.cpu().numpy(), f[idx])
    assert np.array_equal(bo.cpu().numpy(), b[idx])


def test_trainer_prunes_by_view_frequency(abi):
    import torch
    from paper_2403_17898_gb300.render import Trainer, min_count_for
    sc, mlp, _ = synth.CONFIGS["cube4k_128"]()
    views = _views(5, 3)
    tr = Trainer(sc, mlp, 128, 128, track_view_frequency=True)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    tgts = [torch.rand(3, 128, 128, generator=gen, device="cuda") for _ in views]
    tr.train_step(views, tgts)
    # the counts are those of the Trainer's own selections; compare the prune with the oracle
    # rule applied to them
    count = tr.sel_count.cpu().numpy().astype(np.int64)
    assert count.max() <= len(views) and count.sum() > 0
    # the rule applied to the Trainer's own counts (the oracle's form is pinned on its own)
    keep_ref = np.nonzero(~(count / float(len(views)) < 0.4))[0]
    assert min_count_for(len(views), 0.4) == oracle.min_count_for(len(views), 0.4)
    before = {n: getattr(tr, n).cpu().numpy() for n in ("pos", "level", "dL", "feat", "offs", "lv")}
    m_feat = tr.adam_m["feat"].cpu().numpy()
    n = tr.prune(0.4)
    assert n == len(keep_ref) and tr.N == n
    for name, arr in before.items():
        assert np.array_equal(getattr(tr, name).cpu().numpy(), arr[keep_ref]), name
    assert np.array_equal(tr.adam_m["feat"].cpu().numpy(), m_feat[keep_ref])
    tr.train_step(views, tgts)                       # the pruned set still trains
    assert tr.counts().timeout == 0


def test_opacity_accumulate_matches_oracle(abi):
    """Average-opacity statistic (Sec. 4.2.2) over three views against the oracle."""
    import torch
    rng = np.random.default_rng(11)
    N, k, M = 6000, 10, 2500
    acc = torch.zeros(N, device="cuda")
    views = torch.zeros(N, dtype=torch.int32, device="cuda")
    acc_ref = views_ref = None
    for _ in range(3):
        sel = np.sort(rng.choice(N, size=M, replace=False))
        opac = rng.normal(0.1, 0.3, size=M * k).astype(np.float32)   # some dropped (<= 0)
        counts = np.zeros(8, np.uint32)
        counts[0], counts[1] = M, M * k
        abi.opacity_accumulate(cuda(opac), cuda(sel.astype(np.int32)),
                               cuda(counts.view(np.int32)), k, acc, views)
        acc_ref, views_ref = oracle.opacity_accumulate(N, k, sel, opac, acc_ref, views_ref)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(views.cpu().numpy(), views_ref)
    np.testing.assert_allclose(acc.cpu().numpy(), acc_ref, rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("N", [1, 4096, 2_000_000])
def test_prune_by_opacity_matches_oracle(abi, N):
    import torch
    rng = np.random.default_rng(N)
    k = 10
    views = rng.integers(0, 4, size=N)
    acc = (rng.lognormal(np.log(0.01), 1.0, size=N) * views * k).astype(np.float32)
    tau = 0.005
    ref = oracle.prune_by_opacity(acc, views, k, tau)
    keep = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    n_kept = torch.zeros(1, dtype=torch.int32, device="cuda")
    scr = torch.empty(abi.prune_opacity_scratch_bytes(N), dtype=torch.uint8, device="cuda")
    abi.prune_by_opacity(cuda(acc), cuda(views.astype(np.int32)), N, k, tau, keep, n_kept, scr)
    torch.cuda.synchronize()
    n = int(n_kept.item())
    assert n == len(ref)
    assert np.array_equal(keep.cpu().numpy()[:n].astype(np.int64), ref)
    if N > 1:
        assert 0 < n < N


def test_trainer_prunes_by_opacity(abi):
    import torch
    from paper_2403_17898_gb300.render import Trainer
    sc, mlp, _ = synth.CONFIGS["cube4k_128"]()
    views = _views(5, 3)
    tr = Trainer(sc, mlp, 128, 128, track_opacity=True, track_view_frequency=True,
                 track_growth=True)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    tgts = [torch.rand(3, 128, 128, generator=gen, device="cuda") for _ in views]
    tr.train_step(views, tgts)
    s = tr.opac_sum.cpu().numpy()
    v = tr.opac_views.cpu().numpy().astype(np.int64)
    assert v.max() <= len(views) and v.sum() > 0
    assert np.array_equal(v, tr.sel_count.cpu().numpy())   # the same selections counted
    seen = v > 0
    avg = np.where(seen, s / np.maximum(v, 1) / tr.k, np.inf)
    tau = float(np.quantile(avg[seen], 0.3))
    before = {n: getattr(tr, n).cpu().numpy() for n in ("pos", "feat", "offs", "lv")}
    grad_cnt = tr.grad_cnt.cpu().numpy()
    n = tr.prune_opacity(tau)
    # the rule applied to the Trainer's own statistic (the oracle's form is pinned on its own)
    avg32 = np.zeros(len(s), np.float32)
    np.divide(s.astype(np.float32), (v * tr.k).astype(np.float32), out=avg32, where=seen)
    low = seen & (avg32 < np.float32(tau))
    keep = np.nonzero(~low)[0]
    assert n == len(keep) == tr.N and 0 < n < sc.N
    for name, arr in before.items():
        assert np.array_equal(getattr(tr, name).cpu().numpy(), arr[keep]), name
    assert np.array_equal(tr.grad_cnt.cpu().numpy(), grad_cnt[keep])   # statistics follow
    assert not tr.opac_sum.any() and tr.opac_sum.shape[0] == n
    tr.train_step(views, tgts)                            # the pruned set still trains
    assert tr.counts().timeout == 0
