"""FP64 CPU oracle for batched TabNet inference.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
CPU-baseline leg of the benchmark may import this module; the library's
forward pass never calls it and shares no code with it.

What it computes.  The paper deploys a pre-trained TabNet (Sec. I; Sec. II-B;
Sec. IV-A: n_d = n_a = 8, three decision steps) whose per-step sparsemax
feature masks are the audit artefact returned with every prediction
(Sec. III-B; Sec. V-C, where the masks come from deterministic sparsemax
activations).  The paper does not restate TabNet's equations; they come from
the TabNet publication it cites (Arik & Pfister, AAAI 2021).  Written out
for one row, in the order they run here:

  1. e = [x_num, emb_0[x_cat_0], ..., emb_{n_cat-1}[x_cat_{n_cat-1}]]   (D_e)
  2. f = BN0(e)            BN(v) = w * (v - mu) / sqrt(var + eps) + b
  3. feature transformer FT_s (s = 0..n_steps): layers 1..n_shared use FC
     weights shared by every FT, layers after that use FT-specific weights;
     every layer has its own BN per FT.  Layer l:
         u = BN(W x)  (no bias);  g = u[:N] * sigmoid(u[N:])  (GLU);
         x = g for the first layer, else x = (x + g) * sqrt(0.5).
  4. o = FT_0(f); a = o[n_d:]; P = 1; acc = 0; agg = 0
  5. for i = 1..n_steps:
         z   = BN_att_i(W_att_i a) * P
         M_i = sparsemax(z)
         P   = P * (gamma - M_i)
         o   = FT_i(M_i * f);  d = ReLU(o[:n_d]);  a = o[n_d:]
         acc += d;  eta_i = sum(d);  agg += eta_i * M_i
  6. logits = W_f acc + b_f
  7. agg_D[j] = sum of agg over feature j's columns, divided by sum_j agg_D[j]
     (all zeros when that sum is 0).

Readings where the sources are silent (each listed in the design notes):
the step-0 transformer that only feeds the first ``a``; input BN on the
embedded features; no FC biases except the final linear; GLU linear half
first; shared FC weights with per-FT BN; P starts at 1; outputs are raw
logits; the aggregate is reduced to the original features and normalised.

Sparsemax follows Martins & Astudillo (ICML 2016): sort z descending,
k* = max{k : 1 + k z_(k) > sum_{j<=k} z_(j)}, tau = (sum_{j<=k*} z_(j) - 1)/k*,
M = max(z - tau, 0).

All arithmetic is float64; parameters given as float32 arrays are widened
exactly.  Rows are independent, so rows are batched along axis 0 and every
per-row formula is applied to all rows at once.
"""
from __future__ import annotations

import numpy as np


def _f64(a) -> np.ndarray:
    return np.asarray(a, dtype=np.float64)


def batch_norm(v: np.ndarray, bn: dict, eps: float) -> np.ndarray:
    """Inference-mode batch norm with running statistics (unfolded)."""
    return (_f64(bn["weight"]) * (v - _f64(bn["mean"]))
            / np.sqrt(_f64(bn["var"]) + eps) + _f64(bn["bias"]))


def sigmoid(x: np.ndarray) -> np.ndarray:
    return 1.0 / (1.0 + np.exp(-x))


def glu(u: np.ndarray) -> np.ndarray:
    """Gated linear unit: first half times sigmoid of the second half."""
    n = u.shape[-1] // 2
    return u[..., :n] * sigmoid(u[..., n:])


def sparsemax(z: np.ndarray) -> np.ndarray:
    """Euclidean projection of each row of z onto the probability simplex,
    by the sort-and-threshold rule of Martins & Astudillo (2016)."""
    z = _f64(z)
    zs = -np.sort(-z, axis=-1)                       # descending
    cs = np.cumsum(zs, axis=-1)
    k = np.arange(1, z.shape[-1] + 1, dtype=np.float64)
    ok = 1.0 + k * zs > cs                           # support condition
    kstar = np.max(np.where(ok, k, 0.0), axis=-1)    # largest k that holds
    idx = kstar.astype(np.int64) - 1
    tau = (np.take_along_axis(cs, idx[..., None], axis=-1)[..., 0] - 1.0) / kstar
    return np.maximum(z - tau[..., None], 0.0)


def embed(params: dict, x_num, x_cat) -> np.ndarray:
    """Numeric columns first, then each categorical column's embedding row."""
    cols = [_f64(x_num)]
    x_cat = np.asarray(x_cat)
    for j, table in enumerate(params["emb"]):
        idx = x_cat[:, j]
        if np.any(idx < 0) or np.any(idx >= table.shape[0]):
            raise IndexError(f"categorical column {j}: index out of range")
        cols.append(_f64(table)[idx])
    return np.concatenate(cols, axis=1)


def feature_transformer(params: dict, s: int, x: np.ndarray) -> np.ndarray:
    """FT_s: shared layers then step-specific layers, GLU with sqrt(0.5)
    residual from the second layer on."""
    eps = params["bn_eps"]
    ft = params["ft"][s]
    layers = [(w, bn) for w, bn in zip(params["shared_fc"], ft["shared_bn"])]
    layers += [(w, bn) for w, bn in zip(ft["indep_fc"], ft["indep_bn"])]
    for l, (w, bn) in enumerate(layers):
        u = batch_norm(x @ _f64(w).T, bn, eps)
        g = glu(u)
        x = g if l == 0 else (x + g) * np.sqrt(0.5)
    return x


def feature_groups(params: dict):
    """Column range [lo, hi) of every original feature in the embedded row."""
    groups = [(c, c + 1) for c in range(params["n_num"])]
    c = params["n_num"]
    for e in params["cat_emb_dim"]:
        groups.append((c, c + e))
        c += e
    return groups


def aggregate_mask(params: dict, agg: np.ndarray) -> np.ndarray:
    """Reduce the D_e-wide aggregate to the original features, then
    normalise each row to sum 1 (a row whose sum is 0 stays all zero)."""
    agg_d = np.stack([agg[:, lo:hi].sum(axis=1)
                      for lo, hi in feature_groups(params)], axis=1)
    tot = agg_d.sum(axis=1, keepdims=True)
    safe = np.where(tot > 0, tot, 1.0)
    return np.where(tot > 0, agg_d / safe, 0.0)


def forward(params: dict, x_num, x_cat, internals: bool = False):
    """TabNet inference.  Returns (logits [rows, C], masks [rows, n_steps,
    D_e], agg [rows, n_num + n_cat]); with ``internals`` also a dict holding
    the prior after every step, the step importances eta and the embedded,
    normalised input f."""
    eps = params["bn_eps"]
    gamma = float(params["gamma"])
    n_d = params["n_d"]
    e = embed(params, x_num, x_cat)
    f = batch_norm(e, params["bn0"], eps)
    rows, de = f.shape
    o = feature_transformer(params, 0, f)
    a = o[:, n_d:]
    prior = np.ones((rows, de))
    acc = np.zeros((rows, n_d))
    agg = np.zeros((rows, de))
    masks, priors, etas = [], [], []
    for i in range(1, params["n_steps"] + 1):
        att = params["att"][i - 1]
        z = batch_norm(a @ _f64(att["fc"]).T, att["bn"], eps) * prior
        m = sparsemax(z)
        prior = prior * (gamma - m)
        o = feature_transformer(params, i, m * f)
        d = np.maximum(o[:, :n_d], 0.0)
        a = o[:, n_d:]
        acc = acc + d
        eta = d.sum(axis=1)
        agg = agg + eta[:, None] * m
        masks.append(m)
        priors.append(prior)
        etas.append(eta)
    logits = acc @ _f64(params["final_w"]).T + _f64(params["final_b"])
    masks = np.stack(masks, axis=1) if masks else np.zeros((rows, 0, de))
    agg_d = aggregate_mask(params, agg)
    if internals:
        return logits, masks, agg_d, dict(
            prior=np.stack(priors, axis=1) if priors else np.zeros((rows, 0, de)),
            eta=np.stack(etas, axis=1) if etas else np.zeros((rows, 0)),
            f=f, agg_emb=agg)
    return logits, masks, agg_d
