"""The host-buffer entry point pipelines large calls over row chunks.

``tabnet_forward_host`` splits a call into chunks of about 8 MB of outputs
(whole 128-row tiles), each copied in, run and copied out on one of the
handle's four streams in turn.  Every row is computed by the same kernel as
in one device-buffer launch, so the results must be identical bit for bit,
for every combination of requested outputs (which changes the chunk size),
for more chunks than streams, a ragged last chunk, pageable and pinned host
memory, and both kernel families.
"""
import numpy as np
import pytest

from paper_2510_19689_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tabnet_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19689_b300 import tabnet
    return tabnet


def _device_forward(m, x_num, x_cat, masks, agg):
    dev = torch.device("cuda", 0)
    d = m.dims
    rows = x_num.shape[0]
    lg = torch.full((rows, d.n_classes), float("nan"), device=dev)
    mk = torch.full((rows, d.n_steps, d.d_emb), float("nan"), device=dev) if masks else None
    ag = torch.full((rows, d.n_feat), float("nan"), device=dev) if agg else None
    m.forward(torch.from_numpy(x_num).to(dev), torch.from_numpy(x_cat).to(dev), rows, lg, mk, ag)
    torch.cuda.synchronize()
    return (lg.cpu().numpy(), None if mk is None else mk.cpu().numpy(), None if ag is None else ag.cpu().numpy())


# 70,001 rows of the 35-input model: 8 chunks of 9,856 rows with masks and
# the aggregate (848 output bytes per row), 6 with masks only, 2 with the
# aggregate only, and one with logits alone.
@pytest.mark.parametrize("masks,agg", [(True, True), (True, False), (False, True), (False, False)])
@pytest.mark.parametrize("precision", ["bf16x3", "bf16x6", "fp32"])
def test_chunked_host_forward_equals_one_launch(tabnet_mod, precision, masks, agg):
    params = synth.make_params(synth.SPECS["c2"], 31, bn_affine="random")
    x_num, x_cat = synth.make_rows("c2", 70001, seed=32)
    m = tabnet_mod.Model(synth.to_blob(params), precision)
    host = m.forward_host(x_num, x_cat, masks=masks, agg=agg)
    want = _device_forward(m, x_num, x_cat, masks, agg)
    assert m.poll_status() == 0
    m.close()
    for a, b in zip(host, want):
        if b is None:
            assert a is None
        else:
            np.testing.assert_array_equal(a, b)


def test_pinned_buffers_and_repeated_calls(tabnet_mod):
    """Pinned inputs and outputs, two calls of different sizes on one handle
    (the second reuses the streams and the workspace), and a call on a
    caller's stream that already has work queued."""
    params = synth.make_params(synth.SPECS["c2"], 33, bn_affine="random")
    m = tabnet_mod.Model(synth.to_blob(params), "bf16x3")
    d = m.dims
    s = torch.cuda.Stream()
    for rows, seed in ((45000, 34), (20000, 35)):
        x_num, x_cat = synth.make_rows("c2", rows, seed=seed)
        xn = torch.from_numpy(x_num).pin_memory()
        xc = torch.from_numpy(x_cat).pin_memory()
        lg = torch.empty((rows, d.n_classes)).pin_memory()
        mk = torch.empty((rows, d.n_steps, d.d_emb)).pin_memory()
        ag = torch.empty((rows, d.n_feat)).pin_memory()
        with torch.cuda.stream(s):
            busy = torch.randn(4096, 4096, device="cuda")
            busy = busy @ busy                       # work queued ahead on the caller's stream
        L = tabnet_mod.lib()
        tabnet_mod._check(L.tabnet_forward_host(m._h, tabnet_mod._ptr(xn), tabnet_mod._ptr(xc), rows,
                                                tabnet_mod._ptr(lg), tabnet_mod._ptr(mk), tabnet_mod._ptr(ag),
                                                s.cuda_stream), "tabnet_forward_host")
        want = _device_forward(m, x_num, x_cat, True, True)
        np.testing.assert_array_equal(lg.numpy(), want[0])
        np.testing.assert_array_equal(mk.numpy(), want[1])
        np.testing.assert_array_equal(ag.numpy(), want[2])
    assert m.poll_status() == 0
    m.close()
