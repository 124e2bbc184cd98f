"""Pins of the oracle's sparsemax against what the mathematics fixes.

Sparsemax is the Euclidean projection onto the probability simplex
(Martins & Astudillo 2016); the masks it produces are the per-step audit
output of the deployed TabNet (Sec. III-B, Sec. V-C).  None of these checks
reuses the oracle's sort-and-threshold rule: the brute-force search below
tries every support set in exact rational arithmetic.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from oracle.tabnet_oracle import sparsemax
from paper_2510_19689_b300.synth import SplitMix64


def _brute_force(z):
    """Exact projection by trying every support S: tau_S = (sum_S z - 1)/|S|
    is valid iff z_i > tau_S on S and z_i <= tau_S off S.  Returns the list
    of accepted (S, tau) pairs, computed with Fractions."""
    zq = [Fraction(v) for v in z]
    n = len(zq)
    found = []
    for size in range(1, n + 1):
        for S in itertools.combinations(range(n), size):
            tau = (sum(zq[i] for i in S) - 1) / size
            if all(zq[i] > tau for i in S) and all(
                    zq[i] <= tau for i in range(n) if i not in S):
                found.append((set(S), tau))
    return found


def _cases():
    rng = SplitMix64(7)
    out = []
    for n in range(1, 9):
        for _ in range(25):
            out.append(rng.normal(n))                         # generic
            out.append(np.round(rng.normal(n) * 2) / 4)       # many ties
            out.append(rng.normal(n) * 5)                     # large gaps
            out.append(rng.normal(n) * 0.05)                  # near uniform
    out.append(np.array([0.3, 0.3, 0.3, 0.3]))
    out.append(np.array([2.0, 1.0, 0.0]))                     # gap exactly 1
    return out


@pytest.mark.parametrize("z", _cases())
def test_matches_brute_force_support_search(z):
    found = _brute_force(z)
    assert len(found) == 1, "the projection onto the simplex is unique"
    S, tau = found[0]
    exact = np.array([float(max(Fraction(v) - tau, 0)) for v in z])
    m = sparsemax(z[None, :])[0]
    assert set(np.nonzero(m > 0)[0]) == S
    np.testing.assert_allclose(m, exact, rtol=0, atol=1e-14)


def test_two_element_closed_form():
    # n = 2: M_1 = clip((1 + z_1 - z_2) / 2, 0, 1)
    rng = SplitMix64(11)
    z = rng.normal(2000).reshape(1000, 2) * 1.5
    m = sparsemax(z)
    m1 = np.clip((1 + z[:, 0] - z[:, 1]) / 2, 0, 1)
    np.testing.assert_allclose(m[:, 0], m1, atol=1e-15)
    np.testing.assert_allclose(m[:, 1], 1 - m1, atol=1e-15)


def test_simplex_membership_shift_invariance_and_special_cases():
    rng = SplitMix64(12)
    z = rng.normal(500 * 35).reshape(500, 35) * 3
    m = sparsemax(z)
    assert (m >= 0).all()
    np.testing.assert_allclose(m.sum(axis=1), 1.0, atol=1e-13)
    c = rng.normal(500)[:, None] * 10
    np.testing.assert_allclose(sparsemax(z + c), m, atol=1e-12)
    # equal entries give the uniform distribution
    np.testing.assert_allclose(sparsemax(np.full((3, 7), 0.4)), 1 / 7, atol=1e-15)
    # a lead of at least 1 over the runner-up gives a one-hot mask
    z1 = np.array([[3.0, 2.0, 1.5, -1.0], [0.0, -1.0, -1.0, -3.0]])
    np.testing.assert_array_equal(sparsemax(z1), [[1, 0, 0, 0], [1, 0, 0, 0]])


def test_non_expansive():
    # a projection onto a convex set is 1-Lipschitz in the 2-norm
    rng = SplitMix64(13)
    z = rng.normal(400 * 20).reshape(400, 20) * 2
    w = z + rng.normal(400 * 20).reshape(400, 20) * 0.3
    lhs = np.linalg.norm(sparsemax(z) - sparsemax(w), axis=1)
    rhs = np.linalg.norm(z - w, axis=1)
    assert (lhs <= rhs + 1e-12).all()


def test_minimises_distance_over_random_simplex_points():
    # the output is the closest simplex point: no random feasible point
    # (Dirichlet-like) is closer to z
    rng = SplitMix64(14)
    z = rng.normal(50 * 6).reshape(50, 6)
    m = sparsemax(z)
    for r in range(50):
        g = -np.log(1 - rng.uniform(2000 * 6)).reshape(2000, 6)
        pts = g / g.sum(axis=1, keepdims=True)
        d_rand = np.linalg.norm(pts - z[r], axis=1)
        assert np.linalg.norm(m[r] - z[r]) <= d_rand.min() + 1e-12
