"""Pins of the aggregated-mask statistics oracle against hand-built cases."""
import numpy as np

from oracle import mask_stats_oracle as S


def test_one_hot_rows_count_their_feature():
    agg = np.eye(5)[[0, 0, 3, 1, 3, 3]]
    mean, var, frac = S.mask_stats(agg, 1)
    np.testing.assert_allclose(frac, [2 / 6, 1 / 6, 0, 3 / 6, 0])
    np.testing.assert_allclose(mean, frac)            # one-hot: mean = frequency
    np.testing.assert_allclose(var, frac * (1 - frac))  # Bernoulli variance


def test_ties_rank_lower_index_first():
    agg = np.array([[0.25, 0.25, 0.25, 0.25], [0.1, 0.4, 0.4, 0.1]])
    sel = S.topk_sets(agg, 2)
    assert sel.tolist() == [[True, True, False, False], [False, True, True, False]]
    _, _, frac = S.mask_stats(agg, 3)
    np.testing.assert_allclose(frac, [1.0, 1.0, 1.0, 0.0])  # row 2: 0.4, 0.4, then the first 0.1


def test_mean_and_variance_of_known_columns():
    agg = np.array([[1.0, 0.0], [3.0, 0.0], [5.0, 2.0]])
    mean, var, _ = S.mask_stats(agg, 1)
    np.testing.assert_allclose(mean, [3.0, 2 / 3])
    np.testing.assert_allclose(var, [8 / 3, 8 / 9])


def test_agreement_is_one_on_itself_and_counts_overlaps():
    rng = np.random.default_rng(0)
    a = rng.random((50, 12))
    assert S.topk_agreement(a, a, 4) == 1.0
    b = a.copy()
    b[:, 0] = 2.0                 # force feature 0 into every row's top-4 of b
    ov = (S.topk_sets(a, 4) & S.topk_sets(b, 4)).sum(axis=1)
    assert S.topk_agreement(a, b, 4) == ov.sum() / (50 * 4)
    assert (ov >= 3).all()        # forcing one feature in displaces at most one other
