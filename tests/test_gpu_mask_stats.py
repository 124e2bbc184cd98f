"""Aggregated-mask audit statistics on the GPU against their FP64 definitions.

Means and variances are float32 sums (compensated within each of 1,184 row
blocks, pairwise across blocks) of values in [0, 1]: relative error a few
float32 ulps, gated at 1e-5 relative (plus 1e-9 absolute for near-zero
variances).  Top-k fractions and agreements are integer counts over the same
float32 inputs with the same tie rule, so they must match exactly.
"""
import numpy as np
import pytest

from oracle import mask_stats_oracle as S
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


def _rows(rows, d, seed, ties=True):
    rng = np.random.default_rng(seed)
    a = rng.exponential(1.0, size=(rows, d)) * (rng.random((rows, d)) < 0.4)
    a[a.sum(1) == 0, 0] = 1.0
    a = (a / a.sum(1, keepdims=True)).astype(np.float32)
    if ties:
        a[::7, :] = np.float32(1.0 / d)                 # all entries equal
        a[3::11, 1:4] = a[3::11, 1:2]                   # a run of equal entries
    return a


def _check(tabnet_mod, agg, k):
    dev = torch.device("cuda", 0)
    mean, var, frac = tabnet_mod.mask_stats(torch.from_numpy(agg).to(dev), k)
    torch.cuda.synchronize()
    rm, rv, rf = S.mask_stats(agg, k)
    np.testing.assert_allclose(mean.cpu().numpy(), rm, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(var.cpu().numpy(), rv, rtol=1e-5, atol=1e-9)
    counts = np.round(rf * agg.shape[0]).astype(np.int64)
    np.testing.assert_array_equal(frac.cpu().numpy(), (counts / agg.shape[0]).astype(np.float32))


@pytest.mark.parametrize("rows,d,k", [(1, 5, 1), (7, 3, 3), (1000, 14, 3), (65536 + 13, 35, 5), (4099, 100, 10)])
def test_stats_match_definition(tabnet_mod, rows, d, k):
    _check(tabnet_mod, _rows(rows, d, 100 + d), k)


def test_stats_of_real_aggregates_and_agreement_alone_vs_in_a_batch(tabnet_mod):
    """The library's own aggregates for the 35-input model: statistics over
    the batch, and the top-5 agreement between rows run in one launch and the
    same rows run as two separate launches (identical, so 1.0), and against
    the FP64 oracle's aggregates (the masks' audit view survives split-bf16)."""
    dev = torch.device("cuda", 0)
    params = synth.make_params(synth.SPECS["c2"], 77, bn_affine="random")
    xn, xc = synth.make_rows("c2", 3000, seed=78)
    m = tabnet_mod.Model(synth.to_blob(params), "bf16x3")
    _, _, ag = m.run(torch.from_numpy(xn).to(dev), torch.from_numpy(xc).to(dev))
    _, _, ag1 = m.run(torch.from_numpy(xn[:1500]).to(dev), torch.from_numpy(xc[:1500]).to(dev))
    _, _, ag2 = m.run(torch.from_numpy(xn[1500:]).to(dev), torch.from_numpy(xc[1500:]).to(dev))
    torch.cuda.synchronize()
    _check(tabnet_mod, ag.cpu().numpy(), 5)
    same = tabnet_mod.topk_agreement(ag, torch.cat([ag1, ag2]), 5)
    torch.cuda.synchronize()
    assert same.item() == 1.0
    _, _, ra = O.forward(params, xn, xc)
    ref = torch.from_numpy(ra.astype(np.float32)).to(dev)
    got = tabnet_mod.topk_agreement(ag, ref, 5)
    torch.cuda.synchronize()
    want = S.topk_agreement(ag.cpu().numpy(), ra.astype(np.float32), 5)
    assert got.item() == float(np.float32(want)) and want > 0.99
    m.close()


def test_bad_arguments_are_refused(tabnet_mod):
    dev = torch.device("cuda", 0)
    agg = torch.zeros((4, 3), device=dev)
    with pytest.raises(tabnet_mod.TabnetError):
        tabnet_mod.mask_stats(agg, 4)            # k > d
    with pytest.raises(tabnet_mod.TabnetError):
        tabnet_mod.mask_stats(torch.zeros((4, 2000), device=dev), 3)   # d > 1024
