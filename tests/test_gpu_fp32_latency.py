"""The float32 path's two kernels give the same bits.

A float32 call of few rows runs one warp per row (the latency form: a
1,024-row call of the 14-input model would otherwise fill only 32 of the
148 SMs); a larger call runs four lanes per row with rows tiled across the
CTA.  Both compute every output of every layer as the same sequential FMA
chain over k, and every row-level sum (sparsemax, eta, the aggregate total)
as the same four partial sums combined the same way, so a row's logits,
step masks and aggregate must not depend on which kernel ran it: the rows
of small calls are compared bit for bit with the same rows inside one large
call.  Accuracy against the oracle is tested for both forms in
test_gpu_parity.py (its 1,024-row 14-input case takes the warp-per-row
kernel, its larger cases the four-lane one).
"""
import numpy as np
import pytest

from paper_2510_19689_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BIG = 20000                           # above 32 rows per SM: the four-lane kernel
SMALL = [1, 5, 32, 333, 1024, 4000]   # up to 32 rows per SM: the warp-per-row kernel


def _odd_spec():
    # n_d + n_a = 24: the four-lane kernel's per-row (untiled) GLU layer
    return synth.TabNetSpec(n_num=7, cat_card=(5, 9), cat_emb_dim=(1, 2), n_d=12, n_a=12, n_steps=3, gamma=1.3,
                            n_classes=3)


def _rows(spec, name, n, seed):
    if name is not None:
        return synth.make_rows(name, n, seed=seed)
    rng = np.random.default_rng(seed)
    x_num = rng.lognormal(0.0, 1.0, size=(n, spec.n_num)).astype(np.float32)
    x_cat = np.stack([rng.integers(0, c, size=n) for c in spec.cat_card], axis=1).astype(np.int32)
    return x_num, x_cat


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "odd"])
def test_small_calls_equal_large_call_bitwise(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19689_b300 import tabnet
    spec = _odd_spec() if name == "odd" else synth.SPECS[name]
    params = synth.make_params(spec, 300 + len(name), bn_affine="random")
    m = tabnet.Model(synth.to_blob(params), "fp32")
    d = m.dims
    dev = torch.device("cuda", 0)
    x_num, x_cat = _rows(spec, None if name == "odd" else name, BIG, 7)
    xn = torch.from_numpy(np.ascontiguousarray(x_num)).to(dev)
    xc = torch.from_numpy(np.ascontiguousarray(x_cat)).to(dev)

    def call(r0, r, masks=True, agg=True):
        lg = torch.full((r, d.n_classes), float("nan"), device=dev)
        mk = torch.full((r, d.n_steps, d.d_emb), float("nan"), device=dev) if masks else None
        ag = torch.full((r, d.n_feat), float("nan"), device=dev) if agg else None
        m.forward(xn[r0:r0 + r] if d.n_num else None, xc[r0:r0 + r] if d.n_cat else None, r, lg, mk, ag)
        return lg, mk, ag

    big = call(0, BIG)
    torch.cuda.synchronize()
    assert m.poll_status() == 0
    big = [t.cpu().numpy() for t in big]
    assert all(np.isfinite(t).all() for t in big)

    r0 = 0
    for i, r in enumerate(SMALL):
        r0 = (r0 + 7919 * (i + 1)) % (BIG - r)
        masks, agg = i != 2, i != 3       # calls without one output or the other too
        got = call(r0, r, masks, agg)
        torch.cuda.synchronize()
        assert m.poll_status() == 0
        for key, g, b in zip(("logits", "masks", "agg"), got, big):
            if g is None:
                continue
            np.testing.assert_array_equal(g.cpu().numpy(), b[r0:r0 + r], err_msg=f"{name} rows {r0}+{r} {key}")
    m.close()
