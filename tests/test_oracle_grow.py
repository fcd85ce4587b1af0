"""Pins of the oracle's anchor growing and LOD-bias update (Sec. 4.2.1).

Hand cases fix each branch of the level rule (next level above tau[L + 1], same level
between tau[L] and tau[L + 1], nothing below tau[L], no level above the finest), the voxel a
Gaussian proposes (its position pos + O * l_v rounded to the target level's grid points,
the voxel centres of the Eq. for V_L) and the new anchor's position, the occupancy test,
the first-proposal rule for shared voxels, and the accumulated statistic (a 3-4-5
gradient).  The array form is pinned against the loop form on seeded scenes."""
import numpy as np

import oracle
import synth


def _one(level=1, NL=4, g=None, offs=(0.0, 0.0, 0.0), pos=(1.3, 2.7, -0.6), lv=(1.0, 1.0, 1.0),
         k=1):
    pos = np.array([pos], np.float32)
    lev = np.array([level], np.uint8)
    o = np.zeros((1, k, 3), np.float32)
    o[0, 0] = offs
    acc = np.zeros((1, k), np.float32)
    cnt = np.zeros((1, k), np.int64)
    if g is not None:
        acc[0, 0], cnt[0, 0] = 2.0 * g, 2
    return pos, lev, o, np.array([lv], np.float32), acc, cnt


TAU, BIAS = oracle.grow_thresholds(2e-4, 0.2, 4)
VOX = np.array([4.0, 2.0, 1.0, 0.5], np.float32)


def test_thresholds_closed_form():
    assert TAU[0] == np.float32(2e-4)
    np.testing.assert_allclose(TAU[1:] / TAU[:-1], 2.0 ** 0.2, rtol=1e-6)
    np.testing.assert_allclose(BIAS, 0.25 * TAU, rtol=1e-7)


def test_level_rule_branches():
    # anchor of level 1 (spacing 2) at (1.3, 2.7, -0.6): its voxel rint(pos / 2) = (1, 1, 0)
    pos, lev, o, lv, acc, cnt = _one(level=1, g=0.5 * (TAU[1] + TAU[2]), offs=(1.0, 0.0, 0.0))
    # between tau[1] and tau[2]: same level; mu = (2.3, 2.7, -0.6) -> (1, 1, 0): occupied
    p, L, s, par = oracle.grow_anchors(pos, lev, o, lv, acc, cnt, 4, TAU, VOX)
    assert len(p) == 0
    # push the Gaussian one voxel along x: mu = (3.3, 2.7, -0.6) -> (2, 1, 0), a new level-1
    # anchor at the grid point (4, 2, 0)
    o[0, 0] = (2.0, 0.0, 0.0)
    p, L, s, par = oracle.grow_anchors(pos, lev, o, lv, acc, cnt, 4, TAU, VOX)
    assert list(L) == [1] and list(par) == [0]
    np.testing.assert_array_equal(p[0], [4.0, 2.0, 0.0])
    np.testing.assert_array_equal(s[0], [2.0, 2.0, 2.0])
    # above tau[2]: next level (spacing 1): (3.3, 2.7, -0.6) -> (3, 3, -1)
    acc[0, 0] = 2.0 * np.float32(1.01) * TAU[2]
    p, L, s, par = oracle.grow_anchors(pos, lev, o, lv, acc, cnt, 4, TAU, VOX)
    assert list(L) == [2]
    np.testing.assert_array_equal(p[0], [3.0, 3.0, -1.0])
    np.testing.assert_array_equal(s[0], [1.0, 1.0, 1.0])
    # below tau[1]: nothing
    acc[0, 0] = 2.0 * np.float32(0.99) * TAU[1]
    assert len(oracle.grow_anchors(pos, lev, o, lv, acc, cnt, 4, TAU, VOX)[0]) == 0
    # unseen Gaussian: nothing, whatever its sum
    acc[0, 0], cnt[0, 0] = 1.0, 0
    assert len(oracle.grow_anchors(pos, lev, o, lv, acc, cnt, 4, TAU, VOX)[0]) == 0


def test_finest_level_stays():
    pos, lev, o, lv, acc, cnt = _one(level=3, g=1.0, offs=(3.0, 0.0, 0.0))
    p, L, s, par = oracle.grow_anchors(pos, lev, o, lv, acc, cnt, 4, TAU, VOX)
    assert list(L) == [3]                               # no level 4 in a 4-level tree
    # mu = (4.3, 2.7, -0.6) on the 0.5 grid: rint(8.6, 5.4, -1.2) = (9, 5, -1)
    np.testing.assert_array_equal(p[0], [4.5, 2.5, -0.5])


def test_offset_scaled_by_lv():
    pos, lev, o, lv, acc, cnt = _one(level=0, g=0.5 * (TAU[0] + TAU[1]), offs=(1.0, 0.0, 0.0),
                                     lv=(3.0, 1.0, 1.0))
    # mu = (4.3, 2.7, -0.6) on the 4-grid -> (1, 1, 0); the anchor's voxel is (0, 1, 0)
    p, L, s, par = oracle.grow_anchors(pos, lev, o, lv, acc, cnt, 4, TAU, VOX)
    np.testing.assert_array_equal(p[0], [4.0, 4.0, 0.0])


def test_shared_voxel_first_proposal_wins_and_other_levels_do_not_block():
    pos = np.array([[0.1, 0.1, 0.1], [0.3, 0.1, 0.1], [5.0, 0.2, 0.2]], np.float32)
    lev = np.array([2, 2, 1], np.uint8)
    o = np.zeros((3, 2, 3), np.float32)
    o[0, 1] = (1.2, 0.0, 0.0)                  # mu (1.3, .1, .1): level-2 voxel (1, 0, 0)
    o[1, 0] = (1.1, 0.0, 0.0)                  # mu (1.4, .1, .1): the same voxel
    o[2, 0] = (-4.5, 0.0, 0.0)                 # mu (0.5, .2, .2): level-1 voxel (0, 0, 0)
    acc = np.zeros((3, 2), np.float32)
    cnt = np.zeros((3, 2), np.int64)
    g = 0.5 * (TAU[2] + TAU[3])
    for j, i in ((0, 1), (1, 0)):
        acc[j, i], cnt[j, i] = g, 1
    acc[2, 0], cnt[2, 0] = 0.5 * (TAU[1] + TAU[2]), 1
    p, L, s, par = oracle.grow_anchors(pos, lev, o, np.ones((3, 3), np.float32), acc, cnt, 4,
                                       TAU, VOX)
    # proposal 0*2+1 (anchor 0) beats 1*2+0 (anchor 1) for the shared voxel; anchor 2's
    # level-1 voxel (0, 0, 0) is free at level 1 although the level-2 anchors lie inside it
    assert list(par) == [0, 2] and list(L) == [2, 1]
    np.testing.assert_array_equal(p, [[1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])


def test_accumulate_hand_values():
    # 2 anchors selected as [1, 0], k = 2; W = 8, H = 6: du * 4, dv * 3
    drec = np.zeros((4, 9))
    drec[0, :2] = (3.0 / 4.0, 4.0 / 3.0)        # |(3, 4)| = 5 for anchor 1, slot 0
    drec[3, :2] = (0.25, 0.0)                    # 1 for anchor 0, slot 1
    drec[1, :2] = (100.0, 100.0)                 # invisible: ignored
    tiles = np.array([2, 0, 0, 1])
    acc, cnt = oracle.grow_accumulate(2, 2, np.array([1, 0]), drec, tiles, 8, 6)
    np.testing.assert_allclose(acc, [[0.0, 1.0], [5.0, 0.0]], rtol=1e-15)
    np.testing.assert_array_equal(cnt, [[0, 1], [1, 0]])
    acc, cnt = oracle.grow_accumulate(2, 2, np.array([1, 0]), drec, tiles, 8, 6, acc, cnt)
    np.testing.assert_allclose(acc, [[0.0, 2.0], [10.0, 0.0]], rtol=1e-15)
    np.testing.assert_array_equal(cnt, [[0, 2], [2, 0]])


def test_lod_bias_update_hand_cases():
    lev = np.array([0, 1, 1, 2], np.uint8)
    acc = np.zeros((4, 2), np.float32)
    cnt = np.zeros((4, 2), np.int64)
    # anchor 0: mean (3 t + t) / 4 = t > BIAS[0] when t = 1.01 BIAS[0]
    t = np.float32(1.01) * BIAS[0]
    acc[0] = (3 * t, t)
    cnt[0] = (3, 1)
    acc[1] = (0.99 * BIAS[1], 0.0)               # below
    cnt[1] = (1, 0)
    acc[3] = (5.0, 0.0)                          # never counted: unchanged
    dL = np.array([0.0, 0.5, -0.25, 1.0], np.float32)
    out = oracle.lod_bias_update(lev, acc, cnt, BIAS, 0.01, dL)
    np.testing.assert_array_equal(out, np.float32([0.01, 0.5, -0.25, 1.0]))


def test_vectorized_equals_loop_on_seeded_scenes():
    for seed in range(3):
        sc, _, _ = synth.CONFIGS["cube4k_128"]()
        rng = np.random.default_rng(seed)
        N, k = sc.N, sc.k
        cnt = rng.integers(0, 4, size=(N, k))
        acc = (rng.lognormal(np.log(2e-4), 0.6, size=(N, k)) * cnt).astype(np.float32)
        tau, _ = oracle.grow_thresholds(2e-4, 0.2, sc.NL)
        vox = np.asarray(sc.meta["cell"], np.float32)
        a = oracle.grow_anchors(sc.pos, sc.level, sc.offs, sc.lv, acc, cnt, sc.NL, tau, vox)
        b = oracle.grow_anchors_vectorized(sc.pos, sc.level, sc.offs, sc.lv, acc, cnt, sc.NL,
                                           tau, vox)
        assert len(a[0]) > 100
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_same_level_only_when_next_level_disabled():
    pos, lev, o, lv, acc, cnt = _one(level=1, g=1.0, offs=(2.0, 0.0, 0.0))
    p, L, s, par = oracle.grow_anchors(pos, lev, o, lv, acc, cnt, 4, TAU, VOX, next_level=False)
    assert list(L) == [1]                               # above tau[2], yet stays at level 1
    np.testing.assert_array_equal(p[0], [4.0, 2.0, 0.0])
    sc, _, _ = synth.CONFIGS["cube4k_128"]()
    rng = np.random.default_rng(5)
    cnt = rng.integers(0, 3, size=(sc.N, sc.k))
    acc = (rng.lognormal(np.log(3e-4), 0.6, size=(sc.N, sc.k)) * cnt).astype(np.float32)
    tau, _ = oracle.grow_thresholds(2e-4, 0.2, sc.NL)
    vox = np.asarray(sc.meta["cell"], np.float32)
    a = oracle.grow_anchors(sc.pos, sc.level, sc.offs, sc.lv, acc, cnt, sc.NL, tau, vox, False)
    b = oracle.grow_anchors_vectorized(sc.pos, sc.level, sc.offs, sc.lv, acc, cnt, sc.NL, tau,
                                       vox, False)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # every new anchor sits at its parent's level
    assert np.array_equal(a[1], sc.level[a[3]])


def test_progressive_schedule():
    """Sec. 4.3: start at floor(K/2), one more level per stage, N_{i-1} = omega N_i, the
    stage lengths summing to the progressive iterations."""
    st = oracle.progressive_schedule(8, 10_000, 1.5)
    assert [L for _, L in st] == [4, 5, 6, 7]
    starts = [f for f, _ in st] + [10_000]
    n = np.diff(starts).astype(np.float64)
    np.testing.assert_allclose(n[:-1] / n[1:], 1.5, rtol=2e-3)
    assert st[0][0] == 0
    assert oracle.active_level(st, 0) == 4 and oracle.active_level(st, 9_999) == 7
    assert oracle.active_level(st, starts[1] - 1) == 4 and oracle.active_level(st, starts[1]) == 5
    # omega = 1: equal stages; a single level: one stage
    n1 = np.diff([f for f, _ in oracle.progressive_schedule(6, 900, 1.0)] + [900])
    assert list(n1) == [300, 300, 300]
    assert oracle.progressive_schedule(1, 100, 1.5) == [(0, 0)]
