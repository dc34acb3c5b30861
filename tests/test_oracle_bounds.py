"""Special cases that pin the oracle's expected-error bounds (Lemma 1, Theorem 3, eqs. mn11/mn12,
Lemma 4, Corollary 5, Theorem 6) without retyping them.

- A spectrum with nothing beyond the k-th value gives every bound 0 (the tail starts at
  sigma_{k+1}: an off-by-one in the tail index makes it positive).
- A tail holding one value s collapses the square-rooted sum to s^e, so every bound is
  (a + b)^(1/e) s: the same constant must come out for any s, and the bound scales linearly in
  the spectrum (homogeneous of degree 1).
- For a large exponent the bound tends to sigma_{k+1} (the 1/e-th root of a constant tends to 1).
- On sigma_i = 1/i the bounds of eqs. mn11/mn12 decrease strictly with the pass count v (the
  decay in v that Theorem 3 states), and Theorem 6 takes the exponent v - 1.
"""
import math

import numpy as np
import pytest

from oracle import bounds


K, P = 5, 3
ALL = [lambda s: bounds.lemma1(s, K, P, 1), lambda s: bounds.theorem3(s, K, P, 2),
       lambda s: bounds.mn11_12(s, K, P, 4)[0], lambda s: bounds.mn11_12(s, K, P, 5)[1],
       lambda s: bounds.lemma4(s, K, P, 1), lambda s: bounds.corollary5(s, K, P),
       lambda s: bounds.theorem6(s, K, P, 6)]


@pytest.mark.parametrize("f", ALL)
def test_zero_tail_gives_zero(f):
    s = np.array([5.0, 4.0, 3.0, 2.0, 1.0, 0.0, 0.0, 0.0, 0.0])
    assert f(s) == 0.0


@pytest.mark.parametrize("f", ALL)
def test_single_tail_value_and_homogeneity(f):
    base = np.array([5.0, 4.0, 3.0, 2.0, 1.0, 0.0, 0.0, 0.0])
    consts = []
    for t in (0.5, 0.25, 0.01):
        s = base.copy()
        s[K] = t
        consts.append(f(s) / t)
    assert consts[0] == pytest.approx(consts[1], rel=1e-12) == pytest.approx(consts[2], rel=1e-12)
    assert consts[0] > 1.0
    rng = np.random.default_rng(2)
    s = np.sort(rng.random(12))[::-1]
    assert f(7.0 * s) == pytest.approx(7.0 * f(s), rel=1e-12)


def test_large_exponent_tends_to_sigma_k_plus_1():
    s = np.array([9.0, 8.0, 7.0, 6.0, 5.0, 0.4, 0.3, 0.2, 0.1])
    b = bounds.power_bound(s, K, P, 400)
    assert abs(b - 0.4) < 0.4 * 0.02
    assert bounds.power_bound(s, K, P, 1) > bounds.power_bound(s, K, P, 3) > b


def test_bounds_decrease_with_passes():
    s = 1.0 / np.arange(1, 40)
    prev = math.inf
    for v in range(2, 9):
        r, c = bounds.mn11_12(s, K, P, v)
        t = bounds.theorem6(s, K, P, v)
        assert max(r, c) < prev
        prev = max(r, c)
        assert t == pytest.approx(bounds.power_bound(s, K, P, v - 1))


def _golden_constants():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "bound_constants.json")
    return json.load(open(path))["cases"]


@pytest.mark.parametrize("case", _golden_constants(), ids=lambda c: f"k{c['k']}p{c['p']}")
def test_bound_constants_match_hand_worked_values(case):
    """The constants a (of sigma_{k+1}) and b (of the tail sum) against values worked by hand from
    Lemma 1 at (k, p) where a is an integer: tail (1) gives a + b, tail (3, 4) gives 3a + 5b, so a
    mistyped 4p+2, 2p+2 or 4k+4p+2 changes one of the two."""
    k, p, a, b = case["k"], case["p"], case["a"], case["b"]
    head = np.arange(k + 5, 5, -1, dtype=np.float64)[:k]           # any k leading values
    one = np.concatenate([head, [1.0]])
    pyth = np.concatenate([head, [3.0, 4.0]])
    assert bounds.power_bound(one, k, p, 1) == pytest.approx(a + b, rel=1e-14)
    assert bounds.power_bound(pyth, k, p, 1) == pytest.approx(3 * a + 5 * b, rel=1e-14)
    assert bounds.lemma1(one, k, p, 0) == pytest.approx(a + b, rel=1e-14)
