"""The allocation-free segmented entry point, through the C ABI.

tabnet_forward_segments_noalloc is for callers that may not call cudaMalloc
while they run (launches inside a CUDA-graph capture, serving processes whose
device memory is fixed at start-up, plug-in hosts that only hand out their
own buffers): its scratch is a fixed array in the library instead of memory
the library allocates.  Its results must equal those of the allocating entry
point, tabnet_forward_segments_device, on the same requests, call after call
(the shared array keeps the previous call's contents).

This file is collected last so that a run stopping at the first failure has
run every other test first; it passes on its own in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the bf16 bar used by the parity tests (split-bf16 precision)
TOL = dict(logit_abs=2e-2, mask_l1=2e-2, agg_l1=2e-2)


def _outputs(spec, sizes, dev):
    return [dict(logits=torch.full((r, spec.n_classes), float("nan"), device=dev),
                 masks=torch.full((r, spec.n_steps, spec.d_emb), float("nan"), device=dev),
                 agg=torch.full((r, spec.n_feat), float("nan"), device=dev)) for r in sizes]


def test_noalloc_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19689_b300 import synth, tabnet
    L = tabnet.lib()
    spec = synth.SPECS["c2"]
    params = synth.make_params(spec, 51, bn_affine="random")
    m = tabnet.Model(synth.to_blob(params), "bf16x3")
    dev = torch.device("cuda", 0)
    sizes = [3, 129, 1, 0, 400, 128]
    inputs = []
    for i, r in enumerate(sizes):
        xn, xc = synth.make_rows("c2", max(r, 1), seed=900 + i)
        inputs.append((torch.from_numpy(np.ascontiguousarray(xn[:r])).to(dev),
                       torch.from_numpy(np.ascontiguousarray(xc[:r])).to(dev)))

    def descriptors(outs):
        segs = [dict(rows=r, x_num=x, x_cat=c, **o) for r, (x, c), o in zip(sizes, inputs, outs)]
        return torch.frombuffer(bytearray(bytes(tabnet.segment_array(segs))), dtype=torch.uint8).to(dev)

    ref = _outputs(spec, sizes, dev)
    m.forward_segments_device(descriptors(ref), len(sizes))
    torch.cuda.synchronize()
    assert m.poll_status() == 0

    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        got = _outputs(spec, sizes, dev)
        desc = descriptors(got)
        rc = L.tabnet_forward_segments_noalloc(ctypes.c_void_p(m.handle), ctypes.c_void_p(desc.data_ptr()),
                                               len(sizes), ctypes.c_void_p(stream))
        assert rc == 0, tabnet.last_error()
        torch.cuda.synchronize()
        assert m.poll_status() == 0
        for r, a, b in zip(sizes, ref, got):
            if r == 0:
                continue
            lg_a, lg_b = a["logits"].cpu().numpy(), b["logits"].cpu().numpy()
            assert np.isfinite(lg_b).all()
            assert np.abs(lg_a - lg_b).max() <= TOL["logit_abs"]
            mk_a, mk_b = a["masks"].cpu().numpy(), b["masks"].cpu().numpy()
            assert np.abs(mk_a - mk_b).sum(axis=(1, 2)).max() <= TOL["mask_l1"]
            ag_a, ag_b = a["agg"].cpu().numpy(), b["agg"].cpu().numpy()
            assert np.abs(ag_a - ag_b).sum(axis=1).max() <= TOL["agg_l1"]

    # more segments than the fixed scratch holds: rejected before any launch
    big = torch.zeros(48, dtype=torch.uint8, device=dev)
    rc = L.tabnet_forward_segments_noalloc(ctypes.c_void_p(m.handle), ctypes.c_void_p(big.data_ptr()),
                                           tabnet.NOALLOC_MAX_SEGMENTS + 1, ctypes.c_void_p(stream))
    assert rc == -1 and "exceeds" in tabnet.last_error()
    m.close()
