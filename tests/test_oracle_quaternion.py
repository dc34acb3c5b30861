"""Pins for the oracle's quaternion algebra (Section 2) against facts independent of eq. (1)'s
code: the defining unit rules, associativity, multiplicativity of the norm, and two other
matrix representations (complex adjoint and the real 4x4 representation)."""
import json
import os

import numpy as np
import pytest

from oracle import quaternion as Q
from oracle.qsvd import complex_adjoint, real_representation

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand(rng, *shape):
    return rng.standard_normal((4,) + shape)


def test_unit_rules_from_paper():
    g = json.load(open(os.path.join(GOLD, "hamilton_units.json")))
    u = {k: np.array(v, float) for k, v in g["units"].items()}
    for a, b, want in g["products"]:
        np.testing.assert_array_equal(Q.qmul(u[a], u[b]), np.array(want, float), err_msg=f"{a}{b}")
    f = g["triple"]["factors"]
    np.testing.assert_array_equal(Q.qmul(Q.qmul(u[f[0]], u[f[1]]), u[f[2]]), g["triple"]["value"])


def test_associative_and_norm_multiplicative():
    rng = np.random.default_rng(1)
    a, b, c = (_rand(rng, 50) for _ in range(3))
    np.testing.assert_allclose(Q.qmul(Q.qmul(a, b), c), Q.qmul(a, Q.qmul(b, c)), atol=1e-12)
    np.testing.assert_allclose(Q.qnorm(Q.qmul(a, b)), Q.qnorm(a) * Q.qnorm(b), rtol=1e-13)


def test_conjugate_and_inverse():
    rng = np.random.default_rng(2)
    a, b = _rand(rng, 20), _rand(rng, 20)
    np.testing.assert_allclose(Q.qconj(Q.qmul(a, b)), Q.qmul(Q.qconj(b), Q.qconj(a)), atol=1e-12)
    one = Q.qmul(a, Q.qinv(a))
    np.testing.assert_allclose(one, np.stack([np.ones(20), *np.zeros((3, 20))]), atol=1e-13)
    # q q* = |q|^2 (real)
    np.testing.assert_allclose(Q.qmul(a, Q.qconj(a))[0], Q.qnorm(a) ** 2, rtol=1e-13)
    np.testing.assert_allclose(Q.qmul(a, Q.qconj(a))[1:], 0, atol=1e-12)


def test_not_commutative():
    rng = np.random.default_rng(3)
    a, b = _rand(rng, 5), _rand(rng, 5)
    assert np.abs(Q.qmul(a, b) - Q.qmul(b, a)).max() > 1e-3


def test_qmatmul_brute_force():
    rng = np.random.default_rng(4)
    X, Y = _rand(rng, 3, 5), _rand(rng, 5, 2)
    want = np.zeros((4, 3, 2))
    for i in range(3):
        for j in range(2):
            for k in range(5):
                want[:, i, j] += Q.qmul(X[:, i, k], Y[:, k, j])
    np.testing.assert_allclose(Q.qmatmul(X, Y), want, atol=1e-12)


@pytest.mark.parametrize("rep", [complex_adjoint, real_representation])
def test_qmatmul_is_a_representation_homomorphism(rep):
    rng = np.random.default_rng(5)
    X, Y = _rand(rng, 7, 4), _rand(rng, 4, 6)
    np.testing.assert_allclose(rep(Q.qmatmul(X, Y)), rep(X) @ rep(Y), atol=1e-12)


def test_conjugate_transpose():
    rng = np.random.default_rng(6)
    X, Y = _rand(rng, 4, 3), _rand(rng, 3, 5)
    np.testing.assert_allclose(Q.qH(Q.qmatmul(X, Y)), Q.qmatmul(Q.qH(Y), Q.qH(X)), atol=1e-12)
    np.testing.assert_allclose(complex_adjoint(Q.qH(X)), complex_adjoint(X).conj().T, atol=1e-15)
    np.testing.assert_allclose(real_representation(Q.qH(X)), real_representation(X).T, atol=1e-15)
    assert Q.qfro(X) == pytest.approx(np.linalg.norm(real_representation(X)) / 2.0, rel=1e-14)


def test_storage_size_matches_paper_example():
    g = json.load(open(os.path.join(GOLD, "paper_counts.json")))["storage_example"]
    nbytes = 4 * 8 * g["m"] * g["n"]          # four float64 planes
    assert nbytes / 2 ** 30 == pytest.approx(g["approx_gb"], abs=0.01)
