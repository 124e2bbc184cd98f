"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

The method is TabNet inference as the paper deploys it (Sec. IV-A; masks
returned per call, Sec. III-B).  Tolerances:
  * fp32 (FFMA) path and the three-part split (bf16x6) tensor-core path:
    |logit - ref| <= 1e-5 * max(|ref|, 1) (the stated bar).  Masks and the
    aggregate have no stated bar; each nonzero mask entry z - tau carries a
    few units of fp32 rounding of |z| (|z| up to ~100 on the lognormal
    inputs), so the worst rows are those whose support sits next to a
    near-tie.  On these seeded cases the worst per-row mask L1 over all
    steps is 1.1e-4 (fp32, 35-input model) and 5.4e-5 (bf16x6), and the
    worst aggregate L1 1.5e-5 (the aggregate is summed from the fp32 masks
    in both): gated at 2e-4 / 1e-4 for the masks and 5e-5 for the
    aggregate, about 2x the worst case.
  * bf16x3 (split-bf16 tensor-core) path, the stated bf16 bar:
    |logit - ref| <= 2e-2; argmax agreement >= 99.9 %; per-row L1 of the
    mask error summed over all steps <= 2e-2 (every row); aggregate per-row
    L1 <= 2e-2.
  * bf16 (single-rounded operands) path: rounding every weight and every
    activation once to bf16 alone -- emulated exactly in float64 on the CPU
    on these seeded workloads -- gives logit errors up to ~0.1 and per-row
    mask L1 up to ~1 on the 35-input model (the masks are a projection whose
    support flips under small perturbations of near-tied scores), so the
    stated bar is out of reach for single bf16 rounding; this path is gated
    on what that emulation shows, with a 3x margin: |logit - ref| <= 0.3,
    argmax >= 97 % (emulated: 99.6 % on the 100-input model), mean per-row
    mask L1 <= 0.2, 99th-percentile <= 2.
  * every GPU mask row is on the simplex to 5e-5 (>= 0, sums to 1: the fp32
    rounding of z - tau over the support, |z| <= ~100); every aggregate row
    sums to 1 to 1e-5 or is all zero.
"""
import numpy as np
import pytest

from oracle import tabnet_oracle as O
from paper_2510_19689_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {
    "fp32": dict(logit_rel=1e-5, mask_l1=2e-4, agg_l1=5e-5, argmax=1.0),
    "bf16x3": dict(logit_abs=2e-2, mask_l1=2e-2, agg_l1=2e-2, argmax=0.999),
    "bf16": dict(logit_abs=0.3, mask_l1_mean=0.2, mask_l1_p99=2.0, agg_l1_mean=0.2, argmax=0.97),
    # the three-part split is held to the float32 bar
    "bf16x6": dict(logit_rel=1e-5, mask_l1=1e-4, agg_l1=5e-5, argmax=1.0),
}
PRECISIONS = ["fp32", "bf16x3", "bf16", "bf16x6"]


@pytest.fixture(scope="module")
def tabnet_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19689_b300 import tabnet
    return tabnet


def run_gpu(tabnet_mod, blob, precision, x_num, x_cat, masks=True, agg=True):
    m = tabnet_mod.Model(blob, precision)
    dev = torch.device("cuda", 0)
    d = m.dims
    rows = x_num.shape[0]
    xn = torch.from_numpy(x_num).to(dev)
    xc = torch.from_numpy(x_cat).to(dev)
    lg = torch.full((rows, d.n_classes), float("nan"), device=dev)
    mk = torch.full((rows, d.n_steps, d.d_emb), float("nan"), device=dev) if masks else None
    ag = torch.full((rows, d.n_feat), float("nan"), device=dev) if agg else None
    m.forward(xn if d.n_num else None, xc if d.n_cat else None, rows, lg, mk, ag)
    torch.cuda.synchronize()
    status = m.poll_status()
    out = (lg.cpu().numpy(), None if mk is None else mk.cpu().numpy(), None if ag is None else ag.cpu().numpy())
    m.close()
    return out, status


def check(precision, gpu, ref):
    lg, mk, ag = gpu
    rl, rm, ra = ref
    t = TOL[precision]
    assert np.isfinite(lg).all()
    if "logit_rel" in t:
        err = np.abs(lg - rl) / np.maximum(np.abs(rl), 1.0)
        assert err.max() <= t["logit_rel"], f"logit rel err {err.max():.3e}"
    else:
        err = np.abs(lg - rl)
        assert err.max() <= t["logit_abs"], f"logit abs err {err.max():.3e}"
    agree = (lg.argmax(1) == rl.argmax(1)).mean()
    assert agree >= t["argmax"], f"argmax agreement {agree}"
    if mk is not None:
        assert np.isfinite(mk).all()
        assert (mk >= 0).all()
        np.testing.assert_allclose(mk.sum(axis=2), 1.0, atol=5e-5)
        l1 = np.abs(mk - rm).sum(axis=(1, 2))
        if "mask_l1" in t:
            assert l1.max() <= t["mask_l1"], f"mask L1 {l1.max():.3e}"
        else:
            assert l1.mean() <= t["mask_l1_mean"], f"mean mask L1 {l1.mean():.3e}"
            assert np.quantile(l1, 0.99) <= t["mask_l1_p99"], f"p99 mask L1 {np.quantile(l1, 0.99):.3e}"
    if ag is not None:
        assert np.isfinite(ag).all()
        s = ag.sum(axis=1)
        assert np.all((np.abs(s - 1) < 1e-5) | (np.abs(ag).sum(axis=1) == 0))
        l1 = np.abs(ag - ra).sum(axis=1)
        if "agg_l1" in t:
            assert l1.max() <= t["agg_l1"], f"agg L1 {l1.max():.3e}"
        else:
            assert l1.mean() <= t["agg_l1_mean"], f"mean agg L1 {l1.mean():.3e}"


CASES = [("c1", 1024), ("c2", 4096 + 77), ("c3", 1024 + 5)]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("name,rows", CASES)
def test_parity_configs(tabnet_mod, name, rows, precision):
    params = synth.make_params(synth.SPECS[name], synth.weight_seed(name), bn_affine="random")
    x_num, x_cat = synth.make_rows(name, rows)
    if precision == "bf16x6" and name == "c3":
        # n_d + n_a = 128 takes two warpgroups, which the three-part split does not run
        with pytest.raises(tabnet_mod.TabnetError) as e:
            tabnet_mod.Model(synth.to_blob(params), precision)
        assert e.value.code == -6
        return
    gpu, status = run_gpu(tabnet_mod, synth.to_blob(params), precision, x_num, x_cat)
    assert status == 0
    check(precision, gpu, O.forward(params, x_num, x_cat))


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("rows", [1, 2, 127, 128, 129, 300])
def test_ragged_tiles(tabnet_mod, rows, precision):
    params = synth.make_params(synth.SPECS["c2"], 41)
    x_num, x_cat = synth.make_rows("c2", rows, seed=42)
    gpu, status = run_gpu(tabnet_mod, synth.to_blob(params), precision, x_num, x_cat)
    assert status == 0
    check(precision, gpu, O.forward(params, x_num, x_cat))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_optional_outputs_and_zero_rows(tabnet_mod, precision):
    params = synth.make_params(synth.SPECS["c1"], 5)
    blob = synth.to_blob(params)
    x_num, x_cat = synth.make_rows("c1", 200)
    ref = O.forward(params, x_num, x_cat)
    (lg, _, _), st = run_gpu(tabnet_mod, blob, precision, x_num, x_cat, masks=False, agg=False)
    check(precision, (lg, None, None), ref)
    m = tabnet_mod.Model(blob, precision)
    m.forward(None, None, 0, None)  # rows == 0 is a no-op that touches no pointer
    m.close()


# The 100-input model's layout with two steps: its embedded width (160
# columns), A operand, weight ring and shared-memory aggregate leave no room to
# stage the inputs, so the kernel gathers f from global memory at tile start
# and at every step, and the out-of-range check there is exercised too.
WIDE_UNSTAGED = synth.TabNetSpec(n_num=80, cat_card=synth.SPECS["c3"].cat_card, cat_emb_dim=(4,) * 20, n_d=64,
                                 n_a=64, n_steps=2, gamma=1.3, n_classes=3)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("model", ["c1", "wide_unstaged"])
def test_out_of_range_category_sets_status(tabnet_mod, precision, model):
    if model == "c1":
        params = synth.make_params(synth.SPECS["c1"], 6)
        x_num, x_cat = synth.make_rows("c1", 64)
    else:
        if precision in ("fp32", "bf16x6"):
            pytest.skip("fp32 stages nothing and bf16x6 takes n_d + n_a <= 64; covered by the c1 case")
        params = synth.make_params(WIDE_UNSTAGED, 7, bn_affine="random")
        rng = np.random.default_rng(70)
        x_num = rng.lognormal(0.0, 1.0, size=(300, WIDE_UNSTAGED.n_num)).astype(np.float32)
        x_cat = np.stack([rng.integers(0, c, size=300) for c in WIDE_UNSTAGED.cat_card], axis=1).astype(np.int32)
    bad = x_cat.copy()
    bad[5, -1] = 100000
    bad[9, 0] = -3
    bad[len(bad) - 1, 1] = -1
    gpu, status = run_gpu(tabnet_mod, synth.to_blob(params), precision, x_num, bad)
    assert status & 0x1
    # the reference: the same rows with a zero embedding row for those entries
    p2 = dict(params)
    p2["emb"] = [np.vstack([t, np.zeros((1, t.shape[1]), np.float32)]) for t in params["emb"]]
    fixed = bad.copy()
    for j, card in enumerate(params["cat_card"]):
        col = fixed[:, j]
        col[(col < 0) | (col >= card)] = card
    check(precision, gpu, O.forward(p2, x_num, fixed))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_rows_are_independent_bitwise(tabnet_mod, precision):
    """A row's outputs do not depend on the batch around it (same kernel
    configuration): run 700 rows, then a shuffled copy, then single rows."""
    params = synth.make_params(synth.SPECS["c2"], 8)
    blob = synth.to_blob(params)
    x_num, x_cat = synth.make_rows("c2", 700, seed=9)
    (a_lg, a_mk, a_ag), _ = run_gpu(tabnet_mod, blob, precision, x_num, x_cat)
    perm = np.random.default_rng(1).permutation(700)
    (b_lg, b_mk, b_ag), _ = run_gpu(tabnet_mod, blob, precision, x_num[perm], x_cat[perm])
    np.testing.assert_array_equal(a_lg[perm], b_lg)
    np.testing.assert_array_equal(a_mk[perm], b_mk)
    np.testing.assert_array_equal(a_ag[perm], b_ag)
    for r in (0, 333, 699):
        (c_lg, c_mk, c_ag), _ = run_gpu(tabnet_mod, blob, precision, x_num[r:r + 1], x_cat[r:r + 1])
        np.testing.assert_array_equal(a_lg[r:r + 1], c_lg)
        np.testing.assert_array_equal(a_mk[r:r + 1], c_mk)


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_full_size_sampled_rows(tabnet_mod, name):
    """The bench workload at full size in the bench's launch configuration
    (bf16x3, identity BN affine): invariants on every row (checked on the
    device), sampled rows against the oracle."""
    params, blob, x_num, x_cat = synth.load_config(name)
    rows = x_num.shape[0]
    m = tabnet_mod.Model(blob, "bf16x3")
    dev = torch.device("cuda", 0)
    lg, mk, ag = m.run(torch.from_numpy(x_num).to(dev), torch.from_numpy(x_cat).to(dev))
    torch.cuda.synchronize()
    assert m.poll_status() == 0
    m.close()
    assert bool(torch.isfinite(lg).all()) and bool(torch.isfinite(mk).all()) and bool(torch.isfinite(ag).all())
    assert bool((mk >= 0).all())
    assert float((mk.sum(dim=2) - 1).abs().max()) <= 5e-5
    s = ag.sum(dim=1)
    zero_row = ag.abs().sum(dim=1) == 0
    assert bool(((s - 1).abs() < 1e-5).logical_or(zero_row).all())
    idx = np.unique(np.concatenate([np.arange(0, rows, rows // 1500), [rows - 1]]))
    it = torch.from_numpy(idx).to(dev)
    sample = (lg[it].cpu().numpy(), mk[it].cpu().numpy(), ag[it].cpu().numpy())
    del lg, mk, ag
    ref = O.forward(params, x_num[idx], x_cat[idx])
    check("bf16x3", sample, ref)


def test_host_buffer_entry_point(tabnet_mod):
    params = synth.make_params(synth.SPECS["c2"], 12)
    blob = synth.to_blob(params)
    x_num, x_cat = synth.make_rows("c2", 1000, seed=13)
    m = tabnet_mod.Model(blob, "bf16x3")
    host = m.forward_host(x_num, x_cat)
    m.close()
    dev, _ = run_gpu(tabnet_mod, blob, "bf16x3", x_num, x_cat)
    for a, b in zip(host, dev):
        np.testing.assert_array_equal(a, b)


def test_outputs_past_the_int32_element_range(tabnet_mod):
    """1,400,000 rows of the 100-input model in one launch: the step masks
    hold 2.24e9 elements, past 2^31, so every row-offset product must be
    64-bit.  Rows on both sides of mask element 2^31 and the last rows match
    the oracle; every row's masks sum to 1 (checked on the device)."""
    rows = 1_400_000
    spec = synth.SPECS["c3"]
    params = synth.make_params(spec, synth.weight_seed("c3"))
    x_num, x_cat = synth.make_rows("c3", rows, seed=4242)
    m = tabnet_mod.Model(synth.to_blob(params), "bf16x3")
    dev = torch.device("cuda", 0)
    lg, mk, ag = m.run(torch.from_numpy(x_num).to(dev), torch.from_numpy(x_cat).to(dev))
    torch.cuda.synchronize()
    assert m.poll_status() == 0
    m.close()
    per_row = spec.n_steps * spec.d_emb
    assert rows * per_row > 2 ** 31
    assert float((mk.sum(dim=2) - 1).abs().max()) <= 5e-5
    edge = 2 ** 31 // per_row
    idx = np.array([0, edge - 1, edge, edge + 1, rows - 2, rows - 1])
    it = torch.from_numpy(idx).to(dev)
    sample = (lg[it].cpu().numpy(), mk[it].cpu().numpy(), ag[it].cpu().numpy())
    del lg, mk, ag
    check("bf16x3", sample, O.forward(params, x_num[idx], x_cat[idx]))


def test_fp32_width_outside_the_tiled_layer(tabnet_mod):
    """n_d + n_a = 24: the float32 path runs its per-row GLU layer (the
    CTA-wide tiled layer takes widths 16, 32, 64 and 128) and the tensor-core
    modes refuse the width; the float32 results meet the float32 bar."""
    spec = synth.TabNetSpec(n_num=7, cat_card=(5, 9), cat_emb_dim=(1, 2), n_d=12, n_a=12, n_steps=3, gamma=1.3,
                            n_classes=3)
    params = synth.make_params(spec, 90, bn_affine="random")
    rng = np.random.default_rng(91)
    x_num = rng.lognormal(0.0, 1.0, size=(333, spec.n_num)).astype(np.float32)
    x_cat = np.stack([rng.integers(0, c, size=333) for c in spec.cat_card], axis=1).astype(np.int32)
    blob = synth.to_blob(params)
    gpu, status = run_gpu(tabnet_mod, blob, "fp32", x_num, x_cat)
    assert status == 0
    check("fp32", gpu, O.forward(params, x_num, x_cat))
    with pytest.raises(tabnet_mod.TabnetError):
        tabnet_mod.Model(blob, "bf16x3")


def test_wide_model_aggregate_is_summed_in_fp32(tabnet_mod):
    """At 128 hidden units with a 160-column mask (the 100-input model) TMEM
    holds the step mask as fp16 pairs; with the masks requested the
    aggregate is summed from the fp32 mask rows of the output instead.  On
    4,096 seeded rows in split-bf16 the mean per-row aggregate L1 against
    float64 is 1.0e-5 that way and 1.45e-4 from the fp16 copies (2^-11 per
    entry): gated at 4e-5, between the two."""
    params, blob, x_num, x_cat = synth.load_config("c3", rows=4096)
    (lg, mk, ag), st = run_gpu(tabnet_mod, blob, "bf16x3", x_num, x_cat)
    assert st == 0
    ref = O.forward(params, x_num, x_cat)
    agg_l1 = np.abs(ag - ref[2]).sum(axis=1)
    assert agg_l1.mean() <= 4e-5, agg_l1.mean()
    assert agg_l1.max() <= 2e-2
