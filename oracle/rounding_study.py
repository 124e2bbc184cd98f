"""How tensor-core operand roundings move TabNet's outputs (FP64 study).

TEST INFRASTRUCTURE ONLY, under the same rule as ``tabnet_oracle``: only the
tests (and a person running ``python -m oracle.rounding_study``) use it; the
library never does.

``forward_rounded`` is the oracle's forward pass (the step order of
``tabnet_oracle.forward``, reusing its embedding, BN, GLU, sparsemax and
aggregation) in which every fully connected layer -- the GLU layers and the
attentive layers -- multiplies operands rounded the way a tensor-core path
rounds them, with the BN scale folded into the weights first as the library
folds it.  All else (BN shift, GLU, residual, sparsemax, prior, decision,
aggregate, final linear) stays exact float64, so the difference from the
oracle is the effect of the operand rounding alone:

* ``exact``  no rounding (matches the oracle to float64 rounding);
* ``bf16``   weights and FC inputs rounded once to bfloat16 (8 significant
  bits, round to nearest even);
* ``bf16x3`` each operand as hi + lo bfloat16 (lo = bf16(v - hi)) and the
  three products hi*hi + hi*lo + lo*hi accumulated, lo*lo dropped -- what
  three bf16 MMAs per K step compute;
* ``bf16x2w`` / ``bf16x2a`` two of those products: the weight's lo term kept
  (x_hi w_hi + x_hi w_lo) or the activation's (x_hi w_hi + x_lo w_hi) -- what
  two MMAs per K step would compute;
* ``tf32``   both operands rounded to 11 significant bits;
* ``bf16x6`` each operand as three bfloat16 parts (hi, mid = bf16(v - hi),
  lo = bf16(v - hi - mid)) and the six products whose parts' significance
  sums reach 2^-24 (hi hi, hi mid, mid hi, hi lo, mid mid, lo hi);
* ``tf32x3`` each operand as hi + lo in 11-bit significands, three products
  as in ``bf16x3`` -- with ``bf16x6``, the candidates for a tensor-core mode
  at float32 accuracy;
* ``e4m3``   weights scaled per output channel and FC inputs per row to
  amax / 448, rounded to FP8 E4M3 (3 stored mantissa bits, exponent down to
  2^-6, subnormal steps of 2^-9, saturating at 448);
* ``int8``   weights per output channel and FC inputs per row scaled to
  amax / 127 and rounded to the nearest integer (symmetric INT8);
* ``int8w``  weights alone as in ``int8``, FC inputs exact (a weight-only
  INT8 variant, the best any INT8-weight kernel could do).

These tables are why the library's default bf16 mode is split-bf16 with all
three products (it meets the stated bf16 tolerances; neither two-product form
does), and they state the error of its single-rounding modes: plain bf16 and
FP8 E4M3 (whose operands move the sparsemax supports of most rows).  The GPU
tests also hold those two kernels element by element to ``forward_rounded``
in the matching mode.
"""
from __future__ import annotations

import numpy as np

from . import tabnet_oracle as O

MODES = ("exact", "bf16", "bf16x3", "bf16x2w", "bf16x2a", "tf32", "bf16x6", "tf32x3", "e4m3", "int8", "int8w")


def round_significant(x, bits: int) -> np.ndarray:
    """Round to `bits` significant bits, ties to even (no exponent limits)."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(np.ldexp(m, bits)), e - bits)


def round_e4m3(x) -> np.ndarray:
    """Round to the nearest FP8 E4M3 value (ties to even), saturating at 448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, e = np.frexp(a)                    # a = m 2^e with m in [0.5, 1)
    binade = np.maximum(e - 1, -6)        # subnormals share the 2^-6 binade's spacing
    step = np.ldexp(1.0, binade - 3)
    return np.sign(x) * np.minimum(np.rint(a / step) * step, 448.0)


def _parts(v: np.ndarray, bits: int, n: int) -> list:
    """v as n terms of `bits` significant bits: each the rounded remainder."""
    out, rem = [], np.asarray(v, np.float64)
    for _ in range(n):
        t = round_significant(rem, bits)
        out.append(t)
        rem = rem - t
    return out


def _e4m3_scaled(v: np.ndarray, axis: int) -> np.ndarray:
    amax = np.abs(v).max(axis=axis, keepdims=True)
    scale = np.where(amax > 0, amax / 448.0, 1.0)
    return round_e4m3(v / scale) * scale


def _int8_scaled(v: np.ndarray, axis: int) -> np.ndarray:
    amax = np.abs(v).max(axis=axis, keepdims=True)
    scale = np.where(amax > 0, amax / 127.0, 1.0)
    return np.clip(np.rint(v / scale), -127, 127) * scale


def _fc(x: np.ndarray, w, bn: dict, eps: float, mode: str) -> np.ndarray:
    """BN(x W^T) with W's BN scale folded and both operands rounded by `mode`."""
    s = np.asarray(bn["weight"], np.float64) / np.sqrt(np.asarray(bn["var"], np.float64) + eps)
    t = np.asarray(bn["bias"], np.float64) - np.asarray(bn["mean"], np.float64) * s
    ws = s[:, None] * np.asarray(w, np.float64)
    if mode == "exact":
        prod = x @ ws.T
    elif mode == "bf16":
        prod = round_significant(x, 8) @ round_significant(ws, 8).T
    elif mode in ("bf16x3", "bf16x2w", "bf16x2a"):
        xh, wh = round_significant(x, 8), round_significant(ws, 8)
        xl, wl = round_significant(x - xh, 8), round_significant(ws - wh, 8)
        prod = xh @ wh.T
        if mode != "bf16x2a":
            prod = prod + xh @ wl.T
        if mode != "bf16x2w":
            prod = prod + xl @ wh.T
    elif mode == "tf32":
        prod = round_significant(x, 11) @ round_significant(ws, 11).T
    elif mode == "bf16x6":
        xs, wv = _parts(x, 8, 3), _parts(ws, 8, 3)
        prod = sum(xs[i] @ wv[j].T for i, j in ((0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)))
    elif mode == "tf32x3":
        xs, wv = _parts(x, 11, 2), _parts(ws, 11, 2)
        prod = xs[0] @ wv[0].T + xs[0] @ wv[1].T + xs[1] @ wv[0].T
    elif mode == "e4m3":
        prod = _e4m3_scaled(x, axis=1) @ _e4m3_scaled(ws, axis=1).T
    elif mode == "int8":
        prod = _int8_scaled(x, axis=1) @ _int8_scaled(ws, axis=1).T
    elif mode == "int8w":
        prod = x @ _int8_scaled(ws, axis=1).T
    else:
        raise ValueError(f"unknown rounding mode {mode!r}")
    return prod + t


def _feature_transformer(params: dict, s: int, x: np.ndarray, mode: str) -> np.ndarray:
    eps = params["bn_eps"]
    ft = params["ft"][s]
    layers = list(zip(params["shared_fc"], ft["shared_bn"])) + list(zip(ft["indep_fc"], ft["indep_bn"]))
    for l, (w, bn) in enumerate(layers):
        g = O.glu(_fc(x, w, bn, eps, mode))
        x = g if l == 0 else (x + g) * np.sqrt(0.5)
    return x


def forward_rounded(params: dict, x_num, x_cat, mode: str):
    """(logits, masks, agg) of the oracle's forward with rounded FC operands."""
    eps = params["bn_eps"]
    gamma = float(params["gamma"])
    n_d = params["n_d"]
    f = O.batch_norm(O.embed(params, x_num, x_cat), params["bn0"], eps)
    rows, de = f.shape
    o = _feature_transformer(params, 0, f, mode)
    a = o[:, n_d:]
    prior = np.ones((rows, de))
    acc = np.zeros((rows, n_d))
    agg = np.zeros((rows, de))
    masks = []
    for i in range(1, params["n_steps"] + 1):
        att = params["att"][i - 1]
        m = O.sparsemax(_fc(a, att["fc"], att["bn"], eps, mode) * prior)
        prior = prior * (gamma - m)
        o = _feature_transformer(params, i, m * f, mode)
        d = np.maximum(o[:, :n_d], 0.0)
        a = o[:, n_d:]
        acc = acc + d
        agg = agg + d.sum(axis=1)[:, None] * m
        masks.append(m)
    logits = acc @ np.asarray(params["final_w"], np.float64).T + np.asarray(params["final_b"], np.float64)
    return logits, np.stack(masks, axis=1), O.aggregate_mask(params, agg)


def error_summary(ref, got) -> dict:
    """Worst and typical differences of (logits, masks, agg) from the oracle."""
    (rl, rm, ra), (gl, gm, ga) = ref, got
    l1 = np.abs(gm - rm).sum(axis=(1, 2))
    al1 = np.abs(ga - ra).sum(axis=1)
    return dict(logit_max=float(np.abs(gl - rl).max()), argmax=float((gl.argmax(1) == rl.argmax(1)).mean()),
                mask_l1_max=float(l1.max()), mask_l1_p99=float(np.quantile(l1, 0.99)),
                mask_l1_mean=float(l1.mean()), agg_l1_max=float(al1.max()), agg_l1_mean=float(al1.mean()))


def main():
    from paper_2510_19689_b300 import synth
    for name, rows in (("c1", 2000), ("c2", 2000), ("c3", 500)):
        params = synth.make_params(synth.SPECS[name], synth.weight_seed(name), bn_affine="random")
        xn, xc = synth.make_rows(name, rows)
        ref = O.forward(params, xn, xc)
        for mode in MODES[1:]:
            e = error_summary(ref, forward_rounded(params, xn, xc, mode))
            print(f"{name} {rows:5d} rows {mode:7s} logit max {e['logit_max']:.2e}  argmax {e['argmax']:.4f}  "
                  f"mask L1 max/p99/mean {e['mask_l1_max']:.3g} / {e['mask_l1_p99']:.3g} / {e['mask_l1_mean']:.3g}  "
                  f"agg L1 max {e['agg_l1_max']:.3g}", flush=True)


if __name__ == "__main__":
    main()
