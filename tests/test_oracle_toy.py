"""Hand-derived outputs of two tiny TabNets, against the oracle.

The paper prints no worked example of the forward pass (its only numbers are
system measurements on a T4, Sec. V, Tables I-V), so these pins are closed
forms derived by hand from the TabNet definition that the paper deploys
(Sec. IV-A; TabNet of Arik & Pfister 2021).  The derivations are in
``tests/golden/toy_nets.txt``; the expected values below are those closed
forms, with c = 1/sqrt(2).

Toy A: 2 numeric inputs, N = 2, one step, one shared and one step layer,
gamma 1.5, every BN the identity; catches a dropped sqrt(0.5), swapped GLU
halves, a wrong prior or a wrong sparsemax on two entries.

Toy B: 1 numeric + 1 categorical input (embedding dim 2), two steps, gamma
1.2, non-identity input, per-FT and attentive BN, a final bias, one row
whose first decision output is clipped by ReLU and one whose step-1 mask has
full support; catches a BN applied to the wrong FT, a wrong embedding column
order, a missing group sum in the aggregate, eta weighting and a prior
update at the wrong step.
"""
import math

import numpy as np

from oracle import tabnet_oracle as O

C = 1 / math.sqrt(2)


def _bn_id(n, **kw):
    bn = dict(mean=np.zeros(n), var=np.ones(n), weight=np.ones(n), bias=np.zeros(n))
    for k, v in kw.items():
        bn[k] = np.asarray(v, dtype=np.float64)
    return bn


def toy_a():
    eye = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0], [0.0, 0.0]])
    return dict(
        n_num=2, cat_card=[], cat_emb_dim=[], n_d=1, n_a=1, n_steps=1,
        n_shared=1, n_indep=1, n_classes=2, gamma=1.5, bn_eps=0.0,
        emb=[], bn0=_bn_id(2), shared_fc=[eye],
        ft=[dict(shared_bn=[_bn_id(4)], indep_fc=[eye], indep_bn=[_bn_id(4)])
            for _ in range(2)],
        att=[dict(fc=np.array([[0.25], [-0.25]]), bn=_bn_id(2))],
        final_w=np.array([[2.0], [-1.0]]), final_b=np.zeros(2))


def toy_b():
    s2 = math.sqrt(2)
    w_sh = np.array([[1.0, 0, 0], [0, 1, -1], [0, 0, 0], [0, 0, 0]])
    w_ind = np.array([[1.0, 0], [0, -1], [0, 0], [0, 0]])
    ft_bn = [_bn_id(4),
             _bn_id(4, weight=[2, 2, 1, 1], bias=[-0.5, 0, 0, 0]),
             _bn_id(4, bias=[1, 0, 0, 0])]
    return dict(
        n_num=1, cat_card=[3], cat_emb_dim=[2], n_d=1, n_a=1, n_steps=2,
        n_shared=1, n_indep=1, n_classes=2, gamma=1.2, bn_eps=0.0,
        emb=[np.array([[0.0, 0.0], [1.0, -1.0], [3.0, 3.0]])],
        bn0=_bn_id(3, mean=[1, 0, 0], var=[4, 1, 1], weight=[2, 1, 1],
                   bias=[0.5, 0, 0]),
        shared_fc=[w_sh],
        ft=[dict(shared_bn=[ft_bn[s]], indep_fc=[w_ind], indep_bn=[_bn_id(4)])
            for s in range(3)],
        att=[dict(fc=np.array([[2 * s2], [0.0], [-2 * s2]]),
                  bn=_bn_id(3, bias=[0, 0.25, 0])),
             dict(fc=np.array([[16 * s2], [32 * s2], [0.0]]),
                  bn=_bn_id(3, var=[1, 4, 1], bias=[0, 0, 2]))],
        final_w=np.array([[2.0], [-1.0]]), final_b=np.array([0.5, -0.25]))


def test_toy_a_hand_values():
    p = toy_a()
    logits, masks, agg, inn = O.forward(p, np.array([[1.0, 2.0]]),
                                        np.zeros((1, 0), np.int32), internals=True)
    m1 = 0.5 + 3 / (8 * math.sqrt(2))
    d = 9 / 64 + 3 * math.sqrt(2) / 16
    np.testing.assert_allclose(masks[0, 0], [m1, 1 - m1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(inn["prior"][0, 0], [1.5 - m1, 0.5 + m1], atol=1e-14)
    np.testing.assert_allclose(logits[0], [2 * d, -d], atol=1e-14)
    np.testing.assert_allclose(inn["eta"][0], [d], atol=1e-14)
    np.testing.assert_allclose(agg[0], [m1, 1 - m1], atol=1e-14)
    # decimal values of the same closed forms
    np.testing.assert_allclose(masks[0, 0], [0.7651650429449552, 0.2348349570550448], atol=1e-15)
    np.testing.assert_allclose(logits[0], [0.8115800858899107, -0.4057900429449554], atol=1e-15)


def test_toy_b_hand_values():
    p = toy_b()
    x_num = np.array([[2.5], [0.5]])
    x_cat = np.array([[1], [2]], dtype=np.int32)
    logits, masks, agg, inn = O.forward(p, x_num, x_cat, internals=True)
    np.testing.assert_allclose(inn["f"], [[2, 1, -1], [0, 3, 3]], atol=1e-15)
    # row 1
    np.testing.assert_allclose(masks[0], [[0.875, 0.125, 0], [0, 0, 1]], atol=1e-14)
    np.testing.assert_allclose(inn["prior"][0], [[0.325, 1.075, 1.2], [0.39, 1.29, 0.24]], atol=1e-14)
    np.testing.assert_allclose(inn["eta"][0], [2.25 * C, 0.75 * C], atol=1e-14)
    np.testing.assert_allclose(logits[0], [6 * C + 0.5, -3 * C - 0.25], atol=1e-14)
    np.testing.assert_allclose(agg[0], [21 / 32, 11 / 32], atol=1e-14)
    # row 2: first decision output clipped by ReLU, full-support first mask
    np.testing.assert_allclose(masks[1], [[0.25, 0.5, 0.25], [1, 0, 0]], atol=1e-14)
    np.testing.assert_allclose(inn["prior"][1], [[0.95, 0.7, 0.95], [0.19, 0.84, 1.14]], atol=1e-14)
    np.testing.assert_allclose(inn["eta"][1], [0.0, 0.75 * C], atol=1e-14)
    np.testing.assert_allclose(logits[1], [1.5 * C + 0.5, -0.75 * C - 0.25], atol=1e-14)
    np.testing.assert_allclose(agg[1], [1.0, 0.0], atol=1e-14)


def test_zero_weight_model_closed_form():
    """All FC weights zero and every feature-transformer BN with zero mean
    and zero bias: each GLU input is 0, so each GLU output is 0 * sigmoid(0)
    = 0, a = 0 and d = 0; z = BN_att(0) * P, logits = b_f and the
    aggregate is all zeros."""
    from paper_2510_19689_b300 import synth
    p = synth.make_params(synth.SPECS["c1"], 5, bn_affine="random")
    p["shared_fc"] = [np.zeros_like(w) for w in p["shared_fc"]]
    for ft in p["ft"]:
        ft["indep_fc"] = [np.zeros_like(w) for w in ft["indep_fc"]]
        for bn in ft["shared_bn"] + ft["indep_bn"]:
            bn["mean"] = np.zeros_like(bn["mean"])
            bn["bias"] = np.zeros_like(bn["bias"])
    for att in p["att"]:
        att["fc"] = np.zeros_like(att["fc"])
    x_num, x_cat = synth.make_rows("c1", 16)
    logits, masks, agg, inn = O.forward(p, x_num, x_cat, internals=True)
    np.testing.assert_allclose(logits, np.broadcast_to(p["final_b"], logits.shape), atol=1e-7)
    assert (agg == 0).all()
    # the attentive output is the BN shift alone, times the running prior
    prior = np.ones(14)
    for i, att in enumerate(p["att"]):
        bn = att["bn"]
        shift = (bn["bias"].astype(np.float64) - bn["weight"].astype(np.float64)
                 * bn["mean"] / np.sqrt(bn["var"].astype(np.float64) + p["bn_eps"]))
        z = shift * prior
        # for a mask computed from a row-independent z every row agrees
        np.testing.assert_allclose(masks[:, i], np.broadcast_to(masks[0, i], masks[:, i].shape), atol=0)
        assert abs(masks[0, i].sum() - 1) < 1e-12
        # brute force check of this projection
        from tests.test_oracle_sparsemax import _brute_force
        (S, tau), = _brute_force(z)
        np.testing.assert_allclose(masks[0, i], np.maximum(z - float(tau), 0), atol=1e-12)
        prior = prior * (p["gamma"] - masks[0, i])
