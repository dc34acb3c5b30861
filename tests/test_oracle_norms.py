"""Pins for the oracle's spectral norms (the error measure of Lemma 1, Theorems 3 and 6).

Both paths of `oracle.norms.spectral_norm` (LAPACK on the complex adjoint for small matrices,
ARPACK's Lanczos on the implicit quaternion operator for large ones) are checked against closed
forms that do not go through the complex adjoint: a diagonal quaternion matrix has ||D||_2 =
max_i |d_i|, a rank-one u v^H has ||u||·||v||, and a quaternion unitary has norm 1.
"""
import numpy as np

from oracle import norms
from oracle import quaternion as Q


def _rand(rng, *shape):
    return rng.standard_normal((4,) + shape)


def _diag(d):
    n = d.shape[1]
    D = np.zeros((4, n, n))
    D[:, np.arange(n), np.arange(n)] = d
    return D


def test_diagonal_closed_form_dense_and_lanczos():
    rng = np.random.default_rng(11)
    d = _rand(rng, 30)
    d[:, 17] *= 3.0  # a clear maximum, so the Lanczos path converges quickly
    D = _diag(d)
    expect = float(np.sqrt((d * d).sum(axis=0)).max())
    assert abs(norms.spectral_norm(D) - expect) <= 1e-13 * expect
    DH = Q.qH(D)
    got = norms.spectral_norm_op(lambda x: Q.qmatmul(D, x), lambda y: Q.qmatmul(DH, y), 30, 30)
    assert abs(got - expect) <= 1e-9 * expect


def test_rank_one_closed_form_rectangular():
    # ||u v^H||_2 = ||u|| ||v|| for quaternion vectors (the quaternion product is norm-multiplicative
    # entrywise); a transposed operand or a dropped conjugate would break it for non-real entries.
    rng = np.random.default_rng(12)
    u, v = _rand(rng, 23, 1), _rand(rng, 9, 1)
    X = Q.qmatmul(u, Q.qH(v))
    expect = float(np.sqrt((u * u).sum() * (v * v).sum()))
    assert abs(norms.spectral_norm(X) - expect) <= 1e-13 * expect
    XH = Q.qH(X)
    got = norms.spectral_norm_op(lambda x: Q.qmatmul(X, x), lambda y: Q.qmatmul(XH, y), 23, 9)
    assert abs(got - expect) <= 1e-9 * expect


def test_lanczos_path_above_dense_limit():
    # A 1300 x 3 matrix takes the implicit-operator path; its norm equals that of the 3 x 3 Gram's
    # square root, i.e. the largest column norm when the columns are orthogonal by construction.
    rng = np.random.default_rng(13)
    m = 1300
    cols = np.zeros((4, m, 3))
    scale = [5.0, 2.0, 1.0]
    for j in range(3):
        cols[:, 400 * j:400 * j + 300, j] = rng.standard_normal((4, 300))  # disjoint supports
        cols[:, :, j] *= scale[j] / np.sqrt((cols[:, :, j] ** 2).sum())
    assert abs(norms.spectral_norm(cols) - 5.0) <= 1e-9 * 5.0


def test_unitary_has_unit_norm_and_residual_measures():
    rng = np.random.default_rng(14)
    # A quaternion unitary from the oracle's Householder QR of a square matrix.
    from oracle.qr import qr
    Qm, _ = qr(_rand(rng, 12, 12))
    assert abs(norms.spectral_norm(Qm) - 1.0) <= 1e-13
    # X = Q1 B has zero range error against Q1 and a corange error equal to ||X|| when Q2 is
    # orthogonal to X's row space.
    Q1 = Qm[:, :, :5]
    B = _rand(rng, 5, 7)
    X = Q.qmatmul(Q1, B)
    assert norms.range_error(X, Q1) <= 1e-13 * norms.spectral_norm(X)
    Q2 = np.zeros((4, 7, 2))
    Q2[0, 0, 0] = Q2[0, 1, 1] = 1.0
    Xz = X.copy()
    Xz[:, :, :2] = 0.0
    assert abs(norms.corange_error(Xz, Q2) - norms.spectral_norm(Xz)) <= 1e-13 * norms.spectral_norm(Xz)
    assert norms.lowrank_error(X, np.zeros((4, 12, 1)), np.zeros(1), np.zeros((4, 7, 1))) == \
        norms.spectral_norm(X)
