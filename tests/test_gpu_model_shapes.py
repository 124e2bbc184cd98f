"""Model-shape edge cases of the CUDA path against the FP64 oracle.

The workloads all use n_shared = n_indep = 2, gamma > 1 and two or three
classes; the method allows more.  These models each change one degenerate
or boundary property -- no shared layers, no step-specific layers, one
layer per transformer, one decision step, gamma = 1 (a feature used once
has prior 1 - M and can drop out of later masks entirely), one class, the
largest class count of the tensor-core path, numeric-only and
categorical-only inputs, an embedding 192 columns wide (three 64-wide K
blocks in the first layer, the widest the TMEM budget allows at N = 64) --
and must meet each precision's bar of the parity tests on a few ragged
tiles.
"""
import numpy as np
import pytest

from oracle import tabnet_oracle as O
from paper_2510_19689_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BASE = dict(n_num=9, cat_card=(5, 12), cat_emb_dim=(1, 3), n_d=16, n_a=16, n_steps=3, gamma=1.3, n_classes=2)
SHAPES = {
    "no_shared": dict(n_shared=0, n_indep=2),
    "no_indep": dict(n_shared=2, n_indep=0),
    "one_layer": dict(n_shared=1, n_indep=0),
    "one_step": dict(n_steps=1),
    "gamma_one": dict(gamma=1.0, n_steps=4),
    "one_class": dict(n_classes=1),
    "four_classes": dict(n_classes=4),
    "numeric_only": dict(cat_card=(), cat_emb_dim=()),
    "categorical_only": dict(n_num=0, cat_card=(7, 3, 30), cat_emb_dim=(2, 1, 4)),
    "wide_embedding": dict(n_num=136, cat_card=(9, 40), cat_emb_dim=(24, 32), n_d=32, n_a=32, n_steps=2),
}
# fp32 logits: the stated 1e-5 relative bar is for the stated workloads (and
# is met there, tests/test_gpu_parity.py); these random shapes carry no
# stated bar, and float32 FMA chains through every layer on lognormal inputs
# (|f| up to ~100, ~2^-24 relative per operation, a dozen layers) reach
# ~2e-5 relative on the worst of a few hundred rows: gated at 5e-5.
TOL = {"fp32": (5e-5, 5e-4), "bf16x3": (2e-2, 2e-2), "bf16x6": (5e-5, 5e-4)}


@pytest.fixture(scope="module")
def tabnet_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19689_b300 import tabnet
    return tabnet


def _spec(name):
    kw = dict(BASE)
    kw.update(SHAPES[name])
    return synth.TabNetSpec(**kw)


def _rows(spec, rows, seed):
    rng = np.random.default_rng(seed)
    xn = rng.lognormal(0.0, 1.0, size=(rows, spec.n_num)).astype(np.float32)
    xc = (np.stack([rng.integers(0, c, size=rows) for c in spec.cat_card], axis=1).astype(np.int32)
          if spec.cat_card else np.zeros((rows, 0), np.int32))
    return xn, xc


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "bf16x6"])
@pytest.mark.parametrize("name", sorted(SHAPES))
def test_model_shape(tabnet_mod, name, precision):
    spec = _spec(name)
    params = synth.make_params(spec, 500 + sorted(SHAPES).index(name), bn_affine="random")
    if precision == "bf16x6" and name == "wide_embedding":
        # three 64-wide K blocks in three parts (144 KB of A operand) plus a
        # three-slot ring leave no launch shape within shared memory
        with pytest.raises(tabnet_mod.TabnetError) as e:
            tabnet_mod.Model(synth.to_blob(params), precision)
        assert e.value.code == -6 and "shared memory" in str(e.value)
        return
    rows = 2 * 128 + 37
    xn, xc = _rows(spec, rows, 600)
    dev = torch.device("cuda", 0)
    m = tabnet_mod.Model(synth.to_blob(params), precision)
    d = m.dims
    lg = torch.full((rows, d.n_classes), float("nan"), device=dev)
    mk = torch.full((rows, d.n_steps, d.d_emb), float("nan"), device=dev)
    ag = torch.full((rows, d.n_feat), float("nan"), device=dev)
    m.forward(torch.from_numpy(xn).to(dev) if spec.n_num else None,
              torch.from_numpy(xc).to(dev) if spec.cat_card else None, rows, lg, mk, ag)
    torch.cuda.synchronize()
    assert m.poll_status() == 0
    m.close()
    rl, rm, ra = O.forward(params, xn, xc)
    lg, mk, ag = lg.cpu().numpy(), mk.cpu().numpy(), ag.cpu().numpy()
    logit_tol, mask_tol = TOL[precision]
    if precision != "bf16x3":
        assert (np.abs(lg - rl) / np.maximum(np.abs(rl), 1)).max() <= logit_tol
    else:
        assert np.abs(lg - rl).max() <= logit_tol
    assert np.abs(mk - rm).sum(axis=(1, 2)).max() <= mask_tol
    assert np.abs(ag - ra).sum(axis=1).max() <= mask_tol
    np.testing.assert_allclose(mk.sum(axis=2), 1.0, atol=5e-5)
