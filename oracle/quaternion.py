"""Quaternion numbers and matrices as four real planes (Section 2).  Test infrastructure only.

A quaternion q = q0 + q1 i + q2 j + q3 k is stored as q[0..3]; a quaternion matrix
X = X1 + X2 i + X3 j + X4 k (the paper numbers the planes from 1) is a float64 array of
shape (4, rows, cols) holding X1..X4 as planes 0..3.
"""
from __future__ import annotations

import numpy as np


def qmul(q: np.ndarray, p: np.ndarray) -> np.ndarray:
    """Hamilton product q p of (arrays of) quaternions, written out as eq. (1) of Section 2.

    Both arguments have the four components on axis 0; other axes broadcast."""
    q0, q1, q2, q3 = q[0], q[1], q[2], q[3]
    p0, p1, p2, p3 = p[0], p[1], p[2], p[3]
    return np.stack([
        q0 * p0 - q1 * p1 - q2 * p2 - q3 * p3,
        q0 * p1 + q1 * p0 + q2 * p3 - q3 * p2,
        q0 * p2 - q1 * p3 + q2 * p0 + q3 * p1,
        q0 * p3 + q1 * p2 - q2 * p1 + q3 * p0,
    ])


def qconj(q: np.ndarray) -> np.ndarray:
    """Conjugate q* = q0 - q1 i - q2 j - q3 k (Section 2)."""
    out = np.array(q, dtype=np.float64, copy=True)
    out[1:] *= -1.0
    return out


def qnorm(q: np.ndarray) -> np.ndarray:
    """Norm |q| = sqrt(q0^2 + q1^2 + q2^2 + q3^2) (Section 2)."""
    return np.sqrt(np.sum(np.asarray(q, dtype=np.float64) ** 2, axis=0))


def qinv(q: np.ndarray) -> np.ndarray:
    """Inverse q^{-1} = q* / |q|^2 of a non-zero quaternion (Section 2)."""
    return qconj(q) / qnorm(q) ** 2


def qmatmul(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Quaternion matrix product (XY)_{ij} = sum_k x_{ik} y_{kj}.

    Each entry product is the Hamilton product of eq. (1); applying eq. (1) to whole planes
    turns the sum over k into sixteen real matrix products (a library matmul per term)."""
    X0, X1, X2, X3 = X[0], X[1], X[2], X[3]
    Y0, Y1, Y2, Y3 = Y[0], Y[1], Y[2], Y[3]
    return np.stack([
        X0 @ Y0 - X1 @ Y1 - X2 @ Y2 - X3 @ Y3,
        X0 @ Y1 + X1 @ Y0 + X2 @ Y3 - X3 @ Y2,
        X0 @ Y2 - X1 @ Y3 + X2 @ Y0 + X3 @ Y1,
        X0 @ Y3 + X1 @ Y2 - X2 @ Y1 + X3 @ Y0,
    ])


def qH(X: np.ndarray) -> np.ndarray:
    """Conjugate transpose X^H = X1^T - X2^T i - X3^T j - X4^T k (Section 2)."""
    out = np.ascontiguousarray(np.transpose(X, (0, 2, 1)), dtype=np.float64).copy()
    out[1:] *= -1.0
    return out


def qfro(X: np.ndarray) -> float:
    """Frobenius norm ||X||_F = sqrt(sum_ij |x_ij|^2) (Section 2)."""
    return float(np.sqrt(np.sum(np.asarray(X, dtype=np.float64) ** 2)))


def qeye(n: int) -> np.ndarray:
    out = np.zeros((4, n, n))
    out[0] = np.eye(n)
    return out


def qcols(X: np.ndarray, j0: int, j1: int) -> np.ndarray:
    return X[:, :, j0:j1]


def qhstack(blocks) -> np.ndarray:
    """Column concatenation [B1 B2 ...] of quaternion matrices with equal row counts."""
    return np.concatenate(list(blocks), axis=2)
