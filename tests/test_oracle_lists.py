"""Pins of the oracle's per-tile front-to-back lists (Sec. 3.1) and of the stable key sort."""
import numpy as np

import oracle
import synth


def test_tile_lists_brute_force():
    gx, gy = 9, 7
    rect, depth = synth.random_rects_depths(4, 300, gx, gy, max_span=5, equal_depth_frac=0.1)
    start, lst, tie = oracle.tile_lists(rect, depth, gx, gy)
    for ty in range(gy):
        for tx in range(gx):
            t = ty * gx + tx
            got = lst[start[t]:start[t + 1]].tolist()
            want = [g for g in range(len(rect)) if rect[g, 0] <= tx < rect[g, 2]
                    and rect[g, 1] <= ty < rect[g, 3]]
            want.sort(key=lambda g: (float(depth[g]), g))
            assert got == want
    # the total is the sum of rect areas
    area = np.maximum(rect[:, 2] - rect[:, 0], 0) * np.maximum(rect[:, 3] - rect[:, 1], 0)
    assert start[-1] == area.sum()
    # exact depth ties are reported with zero margin exactly in the tiles that hold them
    for t in range(gx * gy):
        d = depth[lst[start[t]:start[t + 1]]]
        assert (tie[t] == 0.0) == (len(np.unique(d)) < len(d))


def test_stable_sort_properties():
    keys, vals = synth.random_sort_keys(0, 5000, bits=13, dup_frac=0.3)
    k2, v2 = oracle.stable_sort_pairs(keys, vals)
    assert np.all(np.diff(k2.astype(np.int64)) >= 0)
    assert sorted(v2.tolist()) == list(range(5000))
    same = np.diff(k2.astype(np.int64)) == 0
    assert np.all(np.diff(v2.astype(np.int64))[same] > 0)      # equal keys keep input order
    assert np.array_equal(keys[v2], k2)
