"""The list comparison used by the full-size GPU parity tests, checked on the CPU against the
oracle's own lists with planted mistakes: it must find the oracle's lists identical, accept a
swap of two entries whose depths tie and a difference confined to knife-edge Gaussians, and
reject a swap across distinct depths, a missing pair and a pair of another Gaussian."""
import copy

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import TIE_MARGIN, compare_tile_lists


@pytest.fixture(scope="module")
def frame():
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    return sc, oracle.render(sc, mlp, cams[0])


def _as_gpu(fr):
    cnt = np.diff(fr.start)
    tr = np.stack([fr.start[:-1], fr.start[1:]], 1)
    tr[cnt == 0] = 0
    return tr, fr.lst.copy()


def _busy_tile(fr):
    t = int(np.argmax(np.diff(fr.start)))
    assert np.diff(fr.start)[t] > 20
    return t


def _key(fr, k, g):
    return int(fr.sel_idx[g // k] * k + g % k)


def test_oracle_lists_are_identical(frame):
    sc, fr = frame
    tr, pg = _as_gpu(fr)
    ident, st = compare_tile_lists(fr, sc.k, fr.sel_idx, tr, pg)
    assert ident.all() and st["pairs"] == len(fr.lst)


def test_swap_across_distinct_depths(frame):
    sc, fr = frame
    tr, pg = _as_gpu(fr)
    t = _busy_tile(fr)
    s = int(fr.start[t])
    d = fr.proj["depth"][pg[s:s + 20]]
    i = s + int(np.argmax(np.abs(np.diff(d)) / d[:-1]))       # a clear depth gap
    assert abs(fr.proj["depth"][pg[i + 1]] / fr.proj["depth"][pg[i]] - 1) > TIE_MARGIN
    pg[i], pg[i + 1] = pg[i + 1], pg[i]
    with pytest.raises(AssertionError):
        compare_tile_lists(fr, sc.k, fr.sel_idx, tr, pg)
    # explained when one of the two is a knife-edge Gaussian (taken out on both sides)
    ident, _ = compare_tile_lists(fr, sc.k, fr.sel_idx, tr, pg, {_key(fr, sc.k, pg[i])})
    assert not ident.reshape(-1)[t] and ident.sum() == ident.size - 1


def test_swap_of_tied_depths(frame):
    sc, fr = frame
    fr = copy.copy(fr)
    fr.proj = dict(fr.proj)
    fr.proj["depth"] = fr.proj["depth"].copy()
    tr, pg = _as_gpu(fr)
    t = _busy_tile(fr)
    s = int(fr.start[t])
    a, b = pg[s + 3], pg[s + 4]
    fr.proj["depth"][b] = fr.proj["depth"][a] * (1 + 0.1 * TIE_MARGIN)   # a near tie
    pg[s + 3], pg[s + 4] = b, a
    ident, _ = compare_tile_lists(fr, sc.k, fr.sel_idx, tr, pg)
    assert not ident.reshape(-1)[t]


def test_missing_or_foreign_pair(frame):
    sc, fr = frame
    tr, pg = _as_gpu(fr)
    t = _busy_tile(fr)
    s = int(fr.start[t])
    foreign = pg.copy()
    inside = set(pg[s:int(fr.start[t + 1])].tolist())
    foreign[s + 2] = next(g for g in range(len(fr.sel_idx) * sc.k) if g not in inside)
    with pytest.raises(AssertionError):
        compare_tile_lists(fr, sc.k, fr.sel_idx, tr, foreign)
    short = tr.copy()
    short[t, 1] -= 1                                  # the tile's last pair is missing
    short[t + 1:] = np.where(short[t + 1:] > 0, short[t + 1:], 0)
    with pytest.raises(AssertionError):
        compare_tile_lists(fr, sc.k, fr.sel_idx, short, pg)
    # a missing pair of a knife-edge Gaussian is explained
    last = int(pg[int(fr.start[t + 1]) - 1])
    cut = np.delete(pg, int(fr.start[t + 1]) - 1)
    cnt = np.diff(fr.start).copy()
    cnt[t] -= 1
    tr2 = np.stack([np.cumsum(cnt) - cnt, np.cumsum(cnt)], 1)
    tr2[cnt == 0] = 0
    ident, _ = compare_tile_lists(fr, sc.k, fr.sel_idx, tr2, cut, {_key(fr, sc.k, last)})
    assert not ident.reshape(-1)[t]


def test_bf16_round_and_gate_model():
    """BF16 rounding: representable values stay, halfway cases go to the even neighbour, the
    rest to the nearest; the gate model equals the FP64 network when inputs, weights and the
    first hidden layer are already representable in BF16."""
    from gpu_helpers import bf16_round, gate_prob_bf16_model
    e = 2.0 ** -7                                      # BF16 spacing just above 1
    x = np.array([1.0, 1.0 + e, 1.0 + e / 2, 1.0 + 3 * e / 2, 1.0 + e / 2 + 2.0 ** -20,
                  -(1.0 + e / 2 + 2.0 ** -20), 0.0], np.float32)
    want = np.array([1.0, 1.0 + e, 1.0, 1.0 + 2 * e, 1.0 + e, -(1.0 + e), 0.0], np.float32)
    np.testing.assert_array_equal(bf16_round(x), want)
    net = synth.proposal_mlp(seed=3)
    for a in net.arrays():
        a[...] = bf16_round(a)
    net.w1[:, 5:] = 0.0                                # hidden units from 5 exact inputs
    net.w2[...] = np.where(np.arange(64)[None, :] < 1, net.w2, 0.0)   # one first-layer unit
    X = bf16_round(np.random.default_rng(0).normal(size=(50, 37)).astype(np.float32))
    X[:, :5] = np.round(X[:, :5] * 4) / 4              # few bits: exact sums in FP32 and BF16
    net.w1[:, :5] = np.round(net.w1[:, :5] * 8) / 8
    net.b1[...] = np.round(net.b1 * 8) / 8
    p, t = oracle.proposal_forward(net, X.astype(np.float64))
    assert np.array_equal(bf16_round(np.maximum(t["a1"], 0).astype(np.float32)),
                          np.maximum(t["a1"], 0).astype(np.float32))
    np.testing.assert_allclose(gate_prob_bf16_model(net, X), p, rtol=1e-12)
