"""Spectral norms of quaternion matrices and of projection residuals.  Test infrastructure only.

||E||_2 of a quaternion matrix equals the largest singular value of its complex adjoint
chi(E) (every singular value of E appears twice there).  Small matrices use LAPACK on chi(E)
directly; large ones run ARPACK's Lanczos bidiagonalisation (scipy.sparse.linalg.svds) on
chi(E) as an implicit operator whose products are quaternion matrix-vector products.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import LinearOperator, svds

from .quaternion import qmatmul, qH
from .qsvd import complex_adjoint

_DENSE_LIMIT = 1200


def _to_complex(x: np.ndarray) -> np.ndarray:
    """First column of chi(x) for a quaternion column vector x (4, n): [xa; -conj(xb)]."""
    return np.concatenate([x[0] + 1j * x[1], -(x[2] - 1j * x[3])])


def _from_complex(c: np.ndarray) -> np.ndarray:
    n = c.shape[0] // 2
    u, w = c[:n], c[n:]
    return np.stack([u.real, u.imag, -w.real, w.imag])


def spectral_norm_op(apply, apply_h, m: int, n: int, tol: float = 1e-10) -> float:
    """Largest singular value of the quaternion operator x -> apply(x) (n -> m columns)."""
    def mv(c):
        c = np.asarray(c).reshape(-1)
        return _to_complex(apply(_from_complex(c)[:, :, None])[:, :, 0])

    def rmv(c):
        c = np.asarray(c).reshape(-1)
        return _to_complex(apply_h(_from_complex(c)[:, :, None])[:, :, 0])

    op = LinearOperator((2 * m, 2 * n), matvec=mv, rmatvec=rmv, dtype=np.complex128)
    s = svds(op, k=1, tol=tol, return_singular_vectors=False, random_state=0)
    return float(np.max(s))


def spectral_norm(E: np.ndarray) -> float:
    """||E||_2 for a quaternion matrix E of shape (4, m, n)."""
    E = np.asarray(E, dtype=np.float64)
    _, m, n = E.shape
    if max(m, n) <= _DENSE_LIMIT:
        return float(np.linalg.svd(complex_adjoint(E), compute_uv=False)[0])
    EH = qH(E)
    return spectral_norm_op(lambda x: qmatmul(E, x), lambda y: qmatmul(EH, y), m, n)


def range_error(X: np.ndarray, Q1: np.ndarray) -> float:
    """||X - Q1 Q1^H X||_2 (the quantity bounded by Lemma 1 and eq. mn11/mn12, first lines)."""
    X = np.asarray(X, dtype=np.float64)
    return spectral_norm(X - qmatmul(Q1, qmatmul(qH(Q1), X)))


def corange_error(X: np.ndarray, Q2: np.ndarray) -> float:
    """||X - X Q2 Q2^H||_2 (Theorem 3 and eq. mn11/mn12, second lines)."""
    X = np.asarray(X, dtype=np.float64)
    return spectral_norm(X - qmatmul(qmatmul(X, Q2), qH(Q2)))


def lowrank_error(X: np.ndarray, U: np.ndarray, S: np.ndarray, V: np.ndarray) -> float:
    """||X - U diag(S) V^H||_2 for the truncated factors."""
    X = np.asarray(X, dtype=np.float64)
    return spectral_norm(X - qmatmul(U * S[None, None, :], qH(V)))
