"""Invariants of the TabNet forward pass, checked on the FP64 oracle.

Each follows from the definition (TabNet as deployed in Sec. IV-A; masks as
the audit output of Sec. III-B) rather than from the oracle's code:
BN folding, the prior's bounds and product form, row independence
(inference BN uses running statistics), the embedding as a one-hot product,
the GLU gate at zero, and the aggregate's normalisation.
"""
import math

import numpy as np
import pytest

from oracle import tabnet_oracle as O
from paper_2510_19689_b300 import synth


@pytest.fixture(scope="module")
def c1_random():
    p = synth.make_params(synth.SPECS["c1"], 77, bn_affine="random")
    x_num, x_cat = synth.make_rows("c1", 300, seed=78)
    return p, x_num, x_cat


def test_bn_folding_identity():
    # BN(W x) == (diag(s) W) x + (b - s mu), s = w / sqrt(var + eps)
    rng = synth.SplitMix64(3)
    W = rng.normal(64 * 35).reshape(64, 35)
    x = rng.normal(50 * 35).reshape(50, 35) * 3
    bn = dict(mean=rng.normal(64), var=rng.uniform_range(64, 0.5, 2.0),
              weight=rng.uniform_range(64, 0.5, 1.5), bias=rng.normal(64))
    eps = 1e-5
    s = bn["weight"] / np.sqrt(bn["var"] + eps)
    folded = x @ (s[:, None] * W).T + (bn["bias"] - s * bn["mean"])
    ref = O.batch_norm(x @ W.T, bn, eps)
    np.testing.assert_allclose(folded, ref, rtol=1e-13, atol=1e-13)


def test_prior_bounds_and_product_form(c1_random):
    p, x_num, x_cat = c1_random
    g = p["gamma"]
    _, masks, _, inn = O.forward(p, x_num, x_cat, internals=True)
    prior = inn["prior"]
    for k in range(1, p["n_steps"] + 1):
        P = prior[:, k - 1]
        assert (P >= (g - 1) ** k - 1e-12).all() and (P <= g ** k + 1e-12).all()
        # the prior is the running product of (gamma - M_i) of the output masks
        np.testing.assert_allclose(P, np.prod(g - masks[:, :k], axis=1), rtol=1e-13)
    # a column that no mask ever selects keeps P = gamma^k exactly
    never = (masks == 0).all(axis=1)
    assert never.any()
    np.testing.assert_array_equal(prior[:, -1][never],
                                  np.prod(np.full(p["n_steps"], g)))


def test_masks_on_simplex_and_aggregate_normalised(c1_random):
    p, x_num, x_cat = c1_random
    _, masks, agg = O.forward(p, x_num, x_cat)
    assert (masks >= 0).all()
    np.testing.assert_allclose(masks.sum(axis=2), 1.0, atol=1e-12)
    s = agg.sum(axis=1)
    assert np.all((np.abs(s - 1) < 1e-12) | (np.abs(agg).sum(axis=1) == 0))
    assert (agg >= 0).all()


def test_rows_are_independent(c1_random):
    # permutation equivariance and batch invariance: running-stat BN makes
    # each row's outputs a function of that row alone
    p, x_num, x_cat = c1_random
    full = O.forward(p, x_num, x_cat)
    perm = np.random.default_rng(0).permutation(x_num.shape[0])
    shuf = O.forward(p, x_num[perm], x_cat[perm])
    for a, b in zip(full, shuf):
        np.testing.assert_allclose(a[perm], b, rtol=1e-12, atol=1e-12)
    for r in (0, 17, 299):
        one = O.forward(p, x_num[r:r + 1], x_cat[r:r + 1])
        for a, b in zip(full, one):
            np.testing.assert_allclose(a[r:r + 1], b, rtol=1e-12, atol=1e-12)


def test_embedding_is_one_hot_product():
    p = synth.make_params(synth.SPECS["c3"], 9)
    x_num, x_cat = synth.make_rows("c3", 64)
    e = O.embed(p, x_num, x_cat)
    col = p["n_num"]
    np.testing.assert_array_equal(e[:, :col], x_num.astype(np.float64))
    for j, table in enumerate(p["emb"]):
        onehot = np.eye(table.shape[0])[x_cat[:, j]]
        np.testing.assert_array_equal(e[:, col:col + table.shape[1]],
                                      onehot @ table.astype(np.float64))
        col += table.shape[1]
    assert col == synth.SPECS["c3"].d_emb
    with pytest.raises(IndexError):
        bad = x_cat.copy()
        bad[3, 19] = 1000
        O.embed(p, x_num, bad)


def test_glu_and_sigmoid():
    # a gate at 0 passes exactly half of the linear half
    u = np.array([[3.0, -2.0, 0.0, 0.0]])
    np.testing.assert_array_equal(O.glu(u), [[1.5, -1.0]])
    x = np.linspace(-30, 30, 601)
    ref = np.array([1 / (1 + np.exp(-np.longdouble(v))) for v in x], dtype=np.longdouble)
    np.testing.assert_allclose(O.sigmoid(x), ref.astype(np.float64), rtol=1e-15, atol=1e-300)


def test_aggregate_groups_and_zero_rows():
    p = dict(n_num=2, cat_emb_dim=[3, 1])
    agg = np.array([[1.0, 0, 2, 2, 0, 3], [0, 0, 0, 0, 0, 0]])
    out = O.aggregate_mask(p, agg)
    np.testing.assert_allclose(out, [[0.125, 0, 0.5, 0.375], [0, 0, 0, 0]])


def test_generator_reference_values():
    # SplitMix64 seeded with 0: first output of the published generator
    assert int(synth.SplitMix64(0).u64(1)[0]) == 0xE220A8397B1DCDAF
    a = synth.make_rows("c2", 1000)
    b = synth.make_rows("c2", 1000)
    np.testing.assert_array_equal(a[0], b[0])
    x_num, x_cat = a
    assert set(np.unique(x_num[:, 13:])) <= {1.0, 2.0, 3.0, 4.0, 5.0}
    assert (x_num[:, :13] > 0).all()
    assert (x_cat >= 0).all() and (x_cat < np.array(synth.SPECS["c2"].cat_card)).all()
    xn3, _ = synth.make_rows("c3", 4000)
    assert 0.04 < (xn3 == 0).mean() < 0.06
