"""FP64 definitions of the aggregated-mask audit statistics.

TEST INFRASTRUCTURE ONLY (same rule as ``tabnet_oracle``).  The paper audits
TabNet's decisions through the aggregated feature masks and asks whether
they stay stable under load (Sec. V-C); these are the plain definitions of
the statistics the library computes on the device over a window of rows of
an aggregate ``agg`` [rows, d]:

* mean[j] = (1/rows) sum_r agg[r, j];  var[j] = (1/rows) sum_r (agg[r, j] - mean[j])^2
* topk_frac[j] = fraction of rows whose k largest entries include j, equal
  entries ranked by the lower index first (a stable descending sort);
* agreement(a, b) = (1/(rows k)) sum_r |topk(a_r) intersect topk(b_r)|.
"""
import numpy as np


def topk_sets(agg: np.ndarray, k: int) -> np.ndarray:
    """Boolean [rows, d]: True where the feature is among the row's k largest."""
    agg = np.asarray(agg)
    order = np.argsort(-agg, axis=1, kind="stable")  # equal entries keep index order
    sel = np.zeros(agg.shape, dtype=bool)
    np.put_along_axis(sel, order[:, :k], True, axis=1)
    return sel


def mask_stats(agg, k: int):
    a = np.asarray(agg, dtype=np.float64)
    mean = a.mean(axis=0)
    var = ((a - mean) ** 2).mean(axis=0)
    frac = topk_sets(agg, k).mean(axis=0)
    return mean, var, frac


def topk_agreement(agg_a, agg_b, k: int) -> float:
    return float((topk_sets(agg_a, k) & topk_sets(agg_b, k)).sum() / (np.asarray(agg_a).shape[0] * k))
