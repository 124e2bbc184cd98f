"""The single-rounding tensor-core modes against their FP64 emulations.

Plain bf16 (every FC operand rounded once to bfloat16) and FP8 E4M3 (weights
scaled per output channel and FC inputs per row to amax / 448, rounded to
E4M3) cannot meet the stated bf16 bar against the exact oracle: their
rounding alone moves the masks (oracle/rounding_study.py).  So each is pinned
twice:

(a) element by element against ``rounding_study.forward_rounded`` in the same
    mode -- the oracle's forward with the FC operands rounded exactly as the
    kernel rounds them (same scales, same round-to-nearest-even, BN scale
    folded into the weights first).  What is left is float32 arithmetic in
    the kernel and operands that sit within about 1e-6 of a rounding
    boundary and round the other way in the kernel (its activations carry
    float32 rounding, the emulation's do not); such a flip moves one product
    by a rounding step, 2^-9 relative in bf16, 2^-4 in E4M3, and bf16's
    boundaries are 16x denser, so its flips are more frequent and smaller.
    The bulk of the rows matches to float32 rounding: the median logit
    difference is gated at 1e-5 relative (measured <= 1.4e-6); the tails at
    about 3x the worst measured on these cases (TOL below).  A wrong scale,
    byte order, dropped product or transposed operand moves the median by
    orders of magnitude.
(b) against the FP64 oracle: the kernel's error must be the rounding's error
    -- the emulation's own error against the oracle on the same rows, with a
    small margin -- which states the mode's error per configuration.
"""
import numpy as np
import pytest

from oracle import rounding_study as R
from oracle import tabnet_oracle as O
from paper_2510_19689_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [("c1", 1024), ("c2", 4096 + 77), ("c3", 1024 + 5)]
EMU = {"bf16": "bf16", "fp8": "e4m3"}


@pytest.fixture(scope="module")
def tabnet_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19689_b300 import tabnet
    return tabnet


def run_gpu(tabnet_mod, params, precision, x_num, x_cat):
    m = tabnet_mod.Model(synth.to_blob(params), precision)
    dev = torch.device("cuda", 0)
    out = m.run(torch.from_numpy(x_num).to(dev), torch.from_numpy(x_cat).to(dev))
    torch.cuda.synchronize()
    status = m.poll_status()
    m.close()
    return tuple(t.cpu().numpy() for t in out), status


# kernel vs its emulation; measured worst over c1 / c2 / c3 in brackets
TOL = {
    # median logit (1.4e-6), p99 (1.0e-3), max (5.5e-3); mean mask L1 (4.5e-3),
    # rows with mask L1 <= 1e-2 (86 %); mean aggregate L1 (5.1e-4)
    "bf16": dict(med=1e-5, p99=3e-3, max=2e-2, mask_mean=1.5e-2, row_l1=1e-2, row_frac=0.75, agg_mean=2e-3),
    # median (4.4e-8), p99 (2.9e-6), max (5.5e-2); mean mask L1 (1.5e-3), rows
    # with mask L1 <= 1e-3 (99.5 %); mean aggregate L1 (2.7e-4)
    "fp8": dict(med=1e-5, p99=1e-4, max=0.15, mask_mean=5e-3, row_l1=1e-3, row_frac=0.97, agg_mean=1e-3),
}


def against_emulation(gpu, emu, precision):
    (lg, mk, ag), (el, em, ea) = gpu, emu
    t = TOL[precision]
    assert np.isfinite(lg).all() and np.isfinite(mk).all() and np.isfinite(ag).all()
    assert (mk >= 0).all()
    np.testing.assert_allclose(mk.sum(axis=2), 1.0, atol=5e-5)
    rel = np.abs(lg - el) / np.maximum(np.abs(el), 1.0)
    assert np.median(rel) <= t["med"], f"logit median {np.median(rel):.3e}"
    assert np.quantile(rel, 0.99) <= t["p99"], f"logit p99 {np.quantile(rel, 0.99):.3e}"
    assert rel.max() <= t["max"], f"logit max {rel.max():.3e}"
    assert (lg.argmax(1) == el.argmax(1)).mean() >= 0.995
    l1 = np.abs(mk - em).sum(axis=(1, 2))
    assert l1.mean() <= t["mask_mean"], f"mean mask L1 {l1.mean():.3e}"
    assert (l1 <= t["row_l1"]).mean() >= t["row_frac"], f"rows within {t['row_l1']}: {(l1 <= t['row_l1']).mean():.4f}"
    al1 = np.abs(ag - ea).sum(axis=1)
    assert al1.mean() <= t["agg_mean"], f"mean agg L1 {al1.mean():.3e}"


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("name,rows", CASES)
def test_tracks_its_emulation(tabnet_mod, name, rows, precision):
    params = synth.make_params(synth.SPECS[name], synth.weight_seed(name), bn_affine="random")
    x_num, x_cat = synth.make_rows(name, rows)
    gpu, status = run_gpu(tabnet_mod, params, precision, x_num, x_cat)
    assert status == 0
    against_emulation(gpu, R.forward_rounded(params, x_num, x_cat, EMU[precision]), precision)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("name,rows", CASES)
def test_error_against_the_oracle_is_the_rounding_error(tabnet_mod, name, rows, precision):
    params = synth.make_params(synth.SPECS[name], synth.weight_seed(name), bn_affine="random")
    x_num, x_cat = synth.make_rows(name, rows)
    gpu, status = run_gpu(tabnet_mod, params, precision, x_num, x_cat)
    assert status == 0
    ref = O.forward(params, x_num, x_cat)
    e_gpu = R.error_summary(ref, gpu)
    e_emu = R.error_summary(ref, R.forward_rounded(params, x_num, x_cat, EMU[precision]))
    assert e_gpu["logit_max"] <= 1.5 * e_emu["logit_max"] + 1e-3, (e_gpu, e_emu)
    assert e_gpu["argmax"] >= e_emu["argmax"] - 0.005, (e_gpu, e_emu)
    assert e_gpu["mask_l1_mean"] <= 1.1 * e_emu["mask_l1_mean"] + 5e-3, (e_gpu, e_emu)
    assert e_gpu["mask_l1_max"] <= 1.5 * e_emu["mask_l1_max"] + 5e-2, (e_gpu, e_emu)
    assert e_gpu["agg_l1_mean"] <= 1.1 * e_emu["agg_l1_mean"] + 5e-3, (e_gpu, e_emu)


@pytest.mark.parametrize("rows", [1, 127, 129, 300])
def test_fp8_ragged_tiles(tabnet_mod, rows):
    params = synth.make_params(synth.SPECS["c2"], 41)
    x_num, x_cat = synth.make_rows("c2", rows, seed=42)
    gpu, status = run_gpu(tabnet_mod, params, "fp8", x_num, x_cat)
    assert status == 0
    emu = R.forward_rounded(params, x_num, x_cat, "e4m3")
    rel = np.abs(gpu[0] - emu[0]) / np.maximum(np.abs(emu[0]), 1.0)
    assert rel.max() <= 0.1 and np.median(rel) <= 1e-5


def test_fp8_rows_are_independent_bitwise(tabnet_mod):
    """The per-row activation scale makes a row's FP8 result depend on its
    own values only: shuffling the batch shuffles the outputs bit for bit."""
    params = synth.make_params(synth.SPECS["c2"], 8)
    x_num, x_cat = synth.make_rows("c2", 700, seed=9)
    a, _ = run_gpu(tabnet_mod, params, "fp8", x_num, x_cat)
    perm = np.random.default_rng(1).permutation(700)
    b, _ = run_gpu(tabnet_mod, params, "fp8", x_num[perm], x_cat[perm])
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x[perm], y)


def test_fp8_full_size_sampled_rows(tabnet_mod):
    """The 100-input workload at full size (1,048,576 rows) in FP8: invariants
    on every row on the device, sampled rows against the E4M3 emulation."""
    params, blob, x_num, x_cat = synth.load_config("c3")
    rows = x_num.shape[0]
    m = tabnet_mod.Model(blob, "fp8")
    dev = torch.device("cuda", 0)
    lg, mk, ag = m.run(torch.from_numpy(x_num).to(dev), torch.from_numpy(x_cat).to(dev))
    torch.cuda.synchronize()
    assert m.poll_status() == 0
    m.close()
    assert bool(torch.isfinite(lg).all()) and bool(torch.isfinite(mk).all()) and bool((mk >= 0).all())
    assert float((mk.sum(dim=2) - 1).abs().max()) <= 5e-5
    idx = np.unique(np.concatenate([np.arange(0, rows, rows // 600), [rows - 1]]))
    it = torch.from_numpy(idx).to(dev)
    sample = (lg[it].cpu().numpy(), mk[it].cpu().numpy(), ag[it].cpu().numpy())
    del lg, mk, ag
    against_emulation(sample, R.forward_rounded(params, x_num[idx], x_cat[idx], "e4m3"), "fp8")
