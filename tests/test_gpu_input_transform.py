"""Preprocessing folded into the model (tabnet_set_input_transform).

A fitted standard scaler (x - mean) * scale on the numeric columns and a
per-column base subtracted from raw categorical codes must give, on raw
inputs, what the model gives on the transformed inputs: checked against the
FP64 oracle run on the transformed inputs, at each precision's bar (the
scaler is folded into the input BN in float32, one more rounding of the
input scale and shift), and the identity transform restores the model
bit for bit.
"""
import numpy as np
import pytest

from oracle import tabnet_oracle as O
from paper_2510_19689_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tabnet_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19689_b300 import tabnet
    return tabnet


def _run(m, xn, xc):
    dev = torch.device("cuda", 0)
    out = m.run(torch.from_numpy(np.ascontiguousarray(xn)).to(dev), torch.from_numpy(np.ascontiguousarray(xc)).to(dev))
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


@pytest.mark.parametrize("precision,logit_tol,mask_tol",
                         [("fp32", 1e-5, 5e-4), ("bf16x3", 2e-2, 2e-2), ("bf16x6", 1e-5, 5e-4)])
@pytest.mark.parametrize("name", ["c1", "c2"])
def test_raw_inputs_through_the_folded_transform(tabnet_mod, name, precision, logit_tol, mask_tol):
    spec = synth.SPECS[name]
    params = synth.make_params(spec, 300, bn_affine="random")
    xn, xc = synth.make_rows(name, 777, seed=301)
    rng = np.random.default_rng(302)
    mean = rng.normal(0, 3, spec.n_num).astype(np.float32)
    scale = np.exp(rng.uniform(-1, 1, spec.n_num)).astype(np.float32)
    base = rng.integers(-5, 1000, spec.n_cat).astype(np.int32)
    raw_n = (xn.astype(np.float64) / scale + mean).astype(np.float32)   # what a caller would hold
    raw_c = xc + base
    m = tabnet_mod.Model(synth.to_blob(params), precision)
    plain = _run(m, xn, xc)
    m.set_input_transform(mean, scale, base)
    got = _run(m, raw_n, raw_c)
    assert m.poll_status() == 0
    ref = O.forward(params, (raw_n.astype(np.float64) - mean) * scale, raw_c - base)
    lg, mk, ag = got
    if precision != "bf16x3":   # the float32 bar: relative
        assert (np.abs(lg - ref[0]) / np.maximum(np.abs(ref[0]), 1)).max() <= logit_tol
    else:
        assert np.abs(lg - ref[0]).max() <= logit_tol
    assert np.abs(mk - ref[1]).sum(axis=(1, 2)).max() <= mask_tol
    assert np.abs(ag - ref[2]).sum(axis=1).max() <= mask_tol
    m.set_input_transform()        # identity again: the model as created
    again = _run(m, xn, xc)
    for a, b in zip(plain, again):
        np.testing.assert_array_equal(a, b)
    m.close()


def test_codes_outside_the_shifted_range_set_the_status(tabnet_mod):
    spec = synth.SPECS["c1"]
    params = synth.make_params(spec, 303)
    xn, xc = synth.make_rows("c1", 64, seed=304)
    m = tabnet_mod.Model(synth.to_blob(params), "bf16x3")
    m.set_input_transform(cat_base=np.full(spec.n_cat, 10, np.int32))
    _run(m, xn, xc)                 # raw codes 0.. are now below every base
    assert m.poll_status() & 1      # TABNET_STATUS_CAT_OOB
    m.close()
