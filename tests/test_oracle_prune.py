"""Pins of the oracle's view-frequency pruning (Sec. 4.2.2): counts are recounted anchor by
anchor, the threshold is applied as "frequency below tau_v is removed"."""
import numpy as np

import oracle
import synth


def test_counts_hand_case():
    sel = [np.array([0, 2, 5]), np.array([2, 5]), np.array([5])]
    np.testing.assert_array_equal(oracle.view_frequency_counts(7, sel), [1, 0, 2, 0, 0, 3, 0])


def test_threshold_hand_cases():
    count = np.array([0, 1, 2, 3, 7, 10])
    # frequency exactly tau_v is kept; below is removed
    np.testing.assert_array_equal(oracle.prune_by_view_frequency(count, 10, 0.7), [4, 5])
    np.testing.assert_array_equal(oracle.prune_by_view_frequency(count, 10, 0.0), range(6))
    assert len(oracle.prune_by_view_frequency(count, 10, 1.01)) == 0
    np.testing.assert_array_equal(oracle.prune_by_view_frequency(count, 10, 0.01), [1, 2, 3, 4, 5])


def test_min_count_matches_the_frequency_test():
    for n in (1, 3, 10, 16, 200, 1000):
        for tau in (0.0, 0.01, 0.2, 0.3, 0.7, 0.7000001, 1.0, 1.2):
            c = oracle.min_count_for(n, tau)
            counts = np.arange(0, n + 2)
            kept = set(oracle.prune_by_view_frequency(counts, n, tau).tolist())
            assert kept == {i for i in counts.tolist() if i >= c}, (n, tau, c)


def test_monotone_in_threshold_and_recount_of_real_selections():
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    rng = np.random.default_rng(4)
    views = [synth.look_at_camera(rng.uniform(-15, 15, 3) + np.array([0, 0, 12.0]),
                                  rng.uniform(-2, 2, 3), 128, 128, d_max=30.0)
             for _ in range(9)]
    sels = [oracle.lod_select(sc.pos, sc.level, sc.dL, sc.NL, v, False)[0] for v in views]
    count = oracle.view_frequency_counts(sc.N, sels)
    for j in rng.choice(sc.N, 50, replace=False):           # brute force, anchor by anchor
        assert count[j] == sum(int(j in set(s.tolist())) for s in sels)
    prev = None
    for tau in (0.0, 0.1, 0.3, 0.5, 0.9, 1.0):
        kept = set(oracle.prune_by_view_frequency(count, len(views), tau).tolist())
        if prev is not None:
            assert kept <= prev
        prev = kept


def test_opacity_statistic_hand_values():
    """Sec. 4.2.2 average opacity: per view, an anchor adds its Gaussians' opacities (dropped
    ones, opacity <= 0, as 0) and one view."""
    opac = np.array([0.5, -0.2, 0.1,    # selected row 0 -> anchor 2: 0.6
                     0.0, 0.3, 0.3])    # selected row 1 -> anchor 0: 0.6
    acc, views = oracle.opacity_accumulate(3, 3, np.array([2, 0]), opac)
    np.testing.assert_allclose(acc, [0.6, 0.0, 0.6], rtol=1e-15)
    np.testing.assert_array_equal(views, [1, 0, 1])
    acc, views = oracle.opacity_accumulate(3, 3, np.array([2]), opac[:3], acc, views)
    np.testing.assert_allclose(acc, [0.6, 0.0, 1.2], rtol=1e-15)
    np.testing.assert_array_equal(views, [1, 0, 2])


def test_prune_by_opacity_threshold():
    k = 10
    acc = np.array([0.05, 0.049, 0.0, 7.0, 0.0], np.float32)
    views = np.array([1, 1, 0, 2, 3])
    # averages 0.005, 0.0049, unseen, 0.35, 0: tau 0.005 keeps the equal one and the unseen
    assert list(oracle.prune_by_opacity(acc, views, k, 0.005)) == [0, 2, 3]
    assert list(oracle.prune_by_opacity(acc, views, k, 0.0)) == [0, 1, 2, 3, 4]
    assert list(oracle.prune_by_opacity(acc, views, k, 1.0)) == [2]
