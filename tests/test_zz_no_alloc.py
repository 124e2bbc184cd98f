"""The allocation-free segmented entry point, through the C ABI.

tabnet_forward_segments_noalloc is for callers that may not call cudaMalloc
once they are running (serving processes whose device memory is fixed at
start-up so that no request can fail or stall on an allocation, plug-in hosts
that only hand out their own buffers): its scratch, the prefix sums of the
segment sizes, is a fixed array in the library instead of memory the library
allocates.  It runs the same kernels with the same prefix sums as the
allocating entry point, tabnet_forward_segments_device, so its results must
equal that entry point's bit for bit, call after call.  The calls here use
different segment lists in turn (the original list, the same sizes
reversed, a short list and a long one), so every call reads prefix-sum
entries that the previous call left different in the shared array: a scan
that skipped rewriting some of them would change the results.

This file is collected last so that a run stopping at the first failure has
run every other test first; it passes on its own in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    stream = torch.cuda.current_stream().cuda_stream
    base = [3, 129, 1, 0, 400, 128]
    lists = [base, base[::-1], [77, 0, 256],
             [int(v) for v in np.random.default_rng(53).integers(0, 40, 301)]]

    for call, sizes in enumerate(lists):
        inputs = []
        for i, r in enumerate(sizes):
            xn, xc = synth.make_rows("c2", max(r, 1), seed=900 + 1000 * call + i)
            inputs.append((torch.from_numpy(np.ascontiguousarray(xn[:r])).to(dev),
                           torch.from_numpy(np.ascontiguousarray(xc[:r])).to(dev)))

        def descriptors(outs):
            segs = [dict(rows=r, x_num=x, x_cat=c, **o) for r, (x, c), o in zip(sizes, inputs, outs)]
            return torch.frombuffer(bytearray(bytes(tabnet.segment_array(segs))), dtype=torch.uint8).to(dev)

        ref = _outputs(spec, sizes, dev)
        m.forward_segments_device(descriptors(ref), len(sizes))
        torch.cuda.synchronize()
        assert m.poll_status() == 0

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
            for key in ("logits", "masks", "agg"):
                x, y = a[key].cpu().numpy(), b[key].cpu().numpy()
                assert np.isfinite(y).all(), (call, r, key)
                np.testing.assert_array_equal(x, y)

    # more segments than the fixed scratch holds: rejected before any launch
    big = torch.zeros(48, dtype=torch.uint8, device=dev)
    rc = L.tabnet_forward_segments_noalloc(ctypes.c_void_p(m.handle), ctypes.c_void_p(big.data_ptr()),
                                           tabnet.NOALLOC_MAX_SEGMENTS + 1, ctypes.c_void_p(stream))
    assert rc == -1 and "exceeds" in tabnet.last_error()
    m.close()
