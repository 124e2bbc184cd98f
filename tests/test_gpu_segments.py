"""Segmented launches (many uneven request batches in one persistent
kernel launch) through the C ABI, against single forwards and the oracle.

The paper sets the batch size per function invocation (Sec. III-B); a
segmented launch serves many invocations at once.  Rows are independent, so
a row's outputs must not depend on which launch, tile or segment mix it ran
in: same launch shape -> bitwise equal to a single forward of its request.
"""
import ctypes

import numpy as np
import pytest

from oracle import tabnet_oracle as O
from paper_2510_19689_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [1, 2, 0, 127, 128, 129, 300, 5, 1000, 64]


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19689_b300 import tabnet
    return tabnet


def _requests(name, sizes, seed):
    dev = torch.device("cuda", 0)
    spec = synth.SPECS[name]
    reqs = []
    for i, r in enumerate(sizes):
        x_num, x_cat = synth.make_rows(name, max(r, 1), seed=seed + i)
        x_num, x_cat = x_num[:r], x_cat[:r]
        reqs.append(dict(
            rows=r, x_num_h=x_num, x_cat_h=x_cat,
            x_num=torch.from_numpy(np.ascontiguousarray(x_num)).to(dev),
            x_cat=torch.from_numpy(np.ascontiguousarray(x_cat)).to(dev),
            logits=torch.full((r, spec.n_classes), float("nan"), device=dev),
            masks=torch.full((r, spec.n_steps, spec.d_emb), float("nan"), device=dev),
            agg=torch.full((r, spec.n_feat), float("nan"), device=dev)))
    return reqs


@pytest.mark.parametrize("precision", ["bf16x3", "bf16", "bf16x6", "fp32"])
def test_segments_equal_single_forwards(tn, precision):
    params = synth.make_params(synth.SPECS["c2"], 31, bn_affine="random")
    m = tn.Model(synth.to_blob(params), precision)
    reqs = _requests("c2", SIZES, 500)
    m.forward_segments(reqs)
    torch.cuda.synchronize()
    assert m.poll_status() == 0
    for q in reqs:
        if q["rows"] == 0:
            continue
        lg, mk, ag = m.run(q["x_num"], q["x_cat"])
        torch.cuda.synchronize()
        assert torch.equal(lg, q["logits"]) and torch.equal(mk, q["masks"]) and torch.equal(ag, q["agg"])
    m.close()


def test_segments_against_oracle(tn):
    params = synth.make_params(synth.SPECS["c3"], 32, bn_affine="random")
    m = tn.Model(synth.to_blob(params), "bf16x3")
    reqs = _requests("c3", [3, 200, 1, 130], 600)
    m.forward_segments(reqs)
    torch.cuda.synchronize()
    for q in reqs:
        rl, rm, ra = O.forward(params, q["x_num_h"], q["x_cat_h"])
        lg, mk, ag = (q[k].cpu().numpy() for k in ("logits", "masks", "agg"))
        assert np.abs(lg - rl).max() <= 2e-2
        assert np.abs(mk - rm).sum(axis=(1, 2)).max() <= 2e-2
        assert np.abs(ag - ra).sum(axis=1).max() <= 2e-2
    m.close()


def test_device_descriptors_in_a_cuda_graph(tn):
    params = synth.make_params(synth.SPECS["c2"], 33)
    m = tn.Model(synth.to_blob(params), "bf16x3")
    reqs = _requests("c2", [77, 1, 400, 129], 700)
    arr = tn.segment_array(reqs)
    dev_desc = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).cuda()
    m.reserve_segments(len(reqs))
    # eager reference
    m.forward_segments_device(dev_desc, len(reqs))
    torch.cuda.synchronize()
    ref = [(q["logits"].clone(), q["masks"].clone(), q["agg"].clone()) for q in reqs]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            m.forward_segments_device(dev_desc, len(reqs), stream=s)
    torch.cuda.synchronize()
    for q in reqs:
        q["logits"].zero_(); q["masks"].zero_(); q["agg"].zero_()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert m.poll_status() == 0
    for q, (lg, mk, ag) in zip(reqs, ref):
        assert torch.equal(q["logits"], lg) and torch.equal(q["masks"], mk) and torch.equal(q["agg"], ag)
    m.close()


def test_segment_argument_errors(tn):
    params = synth.make_params(synth.SPECS["c1"], 34)
    m = tn.Model(synth.to_blob(params), "bf16x3")
    reqs = _requests("c1", [4], 800)
    bad = tn.segment_array(reqs)
    bad[0].rows = -1
    with pytest.raises(tn.TabnetError) as e:
        m.forward_segments(bad)
    assert e.value.code == -1
    bad[0].rows = 4
    bad[0].logits = None
    with pytest.raises(tn.TabnetError):
        m.forward_segments(bad)
    m.forward_segments([])  # zero segments: no launch
    m.close()


def test_uneven_batching_workload_sampled(tn):
    """4,096 request batches of the 35-input model with row counts
    log-uniform in [1, 4096] in one launch (split-bf16): invariants on every
    row, sampled rows of sampled requests against the oracle."""
    params, blob, _, _ = synth.load_config("c2", rows=1)
    sizes = synth.segment_rows(4096, 4096, seed=2004)
    total = int(sizes.sum())
    x_num, x_cat = synth.make_rows("c2", total, seed=2005)
    dev = torch.device("cuda", 0)
    xn = torch.from_numpy(x_num).to(dev)
    xc = torch.from_numpy(x_cat).to(dev)
    spec = synth.SPECS["c2"]
    lg = torch.full((total, spec.n_classes), float("nan"), device=dev)
    mk = torch.full((total, spec.n_steps, spec.d_emb), float("nan"), device=dev)
    ag = torch.full((total, spec.n_feat), float("nan"), device=dev)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    segs = [dict(rows=int(sizes[i]), x_num=xn[offs[i]:], x_cat=xc[offs[i]:], logits=lg[offs[i]:],
                 masks=mk[offs[i]:], agg=ag[offs[i]:]) for i in range(len(sizes))]
    m = tn.Model(blob, "bf16x3")
    m.forward_segments(segs)
    torch.cuda.synchronize()
    assert m.poll_status() == 0
    m.close()
    assert bool(torch.isfinite(lg).all()) and bool(torch.isfinite(mk).all()) and bool(torch.isfinite(ag).all())
    assert float((mk.sum(dim=2) - 1).abs().max()) <= 5e-5
    idx = np.unique(np.concatenate([offs[:-1][::64], offs[1:][::64] - 1, [total - 1]]))
    rl, rm, ra = O.forward(params, x_num[idx], x_cat[idx])
    it = torch.from_numpy(idx).to(dev)
    assert np.abs(lg[it].cpu().numpy() - rl).max() <= 2e-2
    assert np.abs(mk[it].cpu().numpy() - rm).sum(axis=(1, 2)).max() <= 2e-2
    assert np.abs(ag[it].cpu().numpy() - ra).sum(axis=1).max() <= 2e-2
