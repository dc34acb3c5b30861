"""Pins for the oracle's QR (Def. 1, eq. QQR) and QSVD (Def. 1, eq. qsvd)."""
import numpy as np
import pytest

from oracle import quaternion as Q
from oracle.qr import qr
from oracle.qsvd import qsvd, tsvd, singular_values, complex_adjoint, real_representation


def _rand(rng, *shape):
    return rng.standard_normal((4,) + shape)


def _gram_schmidt_bruteforce(Y):
    """Classical Gram-Schmidt with scalar quaternion loops: a second, independent algorithm for
    the unique thin QR with real positive diag(R)."""
    _, m, n = Y.shape
    Qm = np.zeros((4, m, n))
    R = np.zeros((4, n, n))
    for j in range(n):
        v = Y[:, :, j].copy()
        for i in range(j):
            h = np.zeros(4)
            for r in range(m):
                h += Q.qmul(Q.qconj(Qm[:, r, i]), Y[:, r, j])
            R[:, i, j] = h
            for r in range(m):
                v[:, r] -= Q.qmul(Qm[:, r, i], h)
        nv = np.sqrt((v * v).sum())
        R[0, j, j] = nv
        Qm[:, :, j] = v / nv
    return Qm, R


@pytest.mark.parametrize("m,n", [(9, 4), (6, 6), (40, 7)])
def test_qr_factorisation(m, n):
    rng = np.random.default_rng(m * 10 + n)
    Y = _rand(rng, m, n)
    Qm, R = qr(Y)
    np.testing.assert_allclose(Q.qmatmul(Q.qH(Qm), Qm), Q.qeye(n), atol=1e-13)
    np.testing.assert_allclose(Q.qmatmul(Qm, R), Y, atol=1e-12)
    for c in range(4):
        assert np.all(np.tril(R[c], -1) == 0.0)
    d = np.arange(n)
    assert np.all(R[0, d, d] > 0) and np.all(R[1:, d, d] == 0.0)


def test_qr_equals_independent_gram_schmidt():
    rng = np.random.default_rng(11)
    Y = _rand(rng, 8, 5)
    Qm, R = qr(Y)
    Qg, Rg = _gram_schmidt_bruteforce(Y)
    np.testing.assert_allclose(Qm, Qg, atol=1e-12)
    np.testing.assert_allclose(R, Rg, atol=1e-12)


def test_qr_r_is_cholesky_factor_of_gram():
    rng = np.random.default_rng(12)
    Y = _rand(rng, 30, 6)
    _, R = qr(Y)
    np.testing.assert_allclose(Q.qmatmul(Q.qH(R), R), Q.qmatmul(Q.qH(Y), Y), atol=1e-11)


def test_qr_zero_column():
    rng = np.random.default_rng(13)
    Y = _rand(rng, 7, 4)
    Y[:, :, 2] = 0.0
    Qm, R = qr(Y)
    np.testing.assert_allclose(Q.qmatmul(Qm, R), Y, atol=1e-12)
    np.testing.assert_allclose(Q.qmatmul(Q.qH(Qm), Qm), Q.qeye(4), atol=1e-12)
    assert R[0, 2, 2] == 0.0


def test_adjoint_values_come_in_pairs_and_match_real_representation():
    rng = np.random.default_rng(14)
    X = _rand(rng, 9, 6)
    sc = np.linalg.svd(complex_adjoint(X), compute_uv=False)
    np.testing.assert_allclose(sc[0::2], sc[1::2], rtol=1e-12)
    sr = np.linalg.svd(real_representation(X), compute_uv=False)
    for t in range(4):
        np.testing.assert_allclose(sr[t::4], sc[0::2], rtol=1e-12)


def test_qsvd_brute_force_eigen_of_gram():
    """sigma_i^2 are the eigenvalues of X^H X; computed from the real representation of X^H X."""
    rng = np.random.default_rng(15)
    X = _rand(rng, 5, 4)
    s = singular_values(X)
    ev = np.sort(np.linalg.eigvalsh(real_representation(Q.qmatmul(Q.qH(X), X))))[::-1]
    np.testing.assert_allclose(s ** 2, ev[0::4], rtol=1e-12)


@pytest.mark.parametrize("m,n", [(8, 5), (5, 8), (6, 6)])
def test_qsvd_triplets(m, n):
    rng = np.random.default_rng(16 + m + n)
    X = _rand(rng, m, n)
    U, s, V = qsvd(X)
    r = min(m, n)
    assert s.shape == (r,) and np.all(np.diff(s) <= 0)
    np.testing.assert_allclose(Q.qmatmul(Q.qH(U), U), Q.qeye(r), atol=1e-12)
    np.testing.assert_allclose(Q.qmatmul(Q.qH(V), V), Q.qeye(r), atol=1e-12)
    np.testing.assert_allclose(Q.qmatmul(U * s, Q.qH(V)), X, atol=1e-12)
    np.testing.assert_allclose(Q.qmatmul(Q.qH(X), U), V * s, atol=1e-12)   # X^H u = sigma v


def test_qsvd_closed_forms():
    rng = np.random.default_rng(17)
    q = _rand(rng, 1, 1)
    assert singular_values(q)[0] == pytest.approx(Q.qnorm(q[:, 0, 0]), rel=1e-14)
    d = _rand(rng, 5)
    D = np.zeros((4, 5, 5))
    D[:, np.arange(5), np.arange(5)] = d
    np.testing.assert_allclose(singular_values(D), np.sort(Q.qnorm(d))[::-1], rtol=1e-13)


def test_qsvd_repeated_singular_values():
    """A doubled quaternion singular value (a 4-dimensional complex singular subspace) still
    yields an orthonormal quaternion basis (the Gram-Schmidt guard)."""
    rng = np.random.default_rng(18)
    Uq, _ = qr(_rand(rng, 7, 3))
    Vq, _ = qr(_rand(rng, 5, 3))
    s = np.array([1.0, 1.0, 0.5])
    X = Q.qmatmul(Uq * s, Q.qH(Vq))
    U, sv, V = qsvd(X, rank=3)
    np.testing.assert_allclose(sv, s, rtol=1e-12)
    np.testing.assert_allclose(Q.qmatmul(Q.qH(V), V), Q.qeye(3), atol=1e-12)
    np.testing.assert_allclose(Q.qmatmul(U * sv, Q.qH(V)), X, atol=1e-12)


def test_tsvd_truncates():
    rng = np.random.default_rng(19)
    R = _rand(rng, 6, 6)
    L, s, Rt = tsvd(R, 3)
    assert L.shape == (4, 6, 3) and Rt.shape == (4, 6, 3)
    np.testing.assert_allclose(s, singular_values(R)[:3], rtol=1e-12)
    np.testing.assert_allclose(Q.qmatmul(R, Rt), L * s, atol=1e-12)
