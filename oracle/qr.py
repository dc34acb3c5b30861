"""Thin quaternion QR by Householder reflections (Def. 1, eq. QQR).  Test infrastructure only.

The paper's QR has no sign or phase convention.  The oracle returns the thin factorisation
Y = Q R with Q^H Q = I and R upper triangular whose diagonal is real and non-negative.  For a
full-column-rank Y this factorisation is unique, so any correct QR (Householder here,
CholeskyQR2 on the GPU) must agree with it up to rounding.
"""
from __future__ import annotations

import numpy as np

from .quaternion import qmatmul, qH, qnorm, qconj, qmul


def householder_qr(Y: np.ndarray):
    """Return (Q, R) with Y = Q R for a quaternion matrix Y of shape (4, m, n), m >= n.

    Step j reflects the trailing part x of column j onto a multiple of e_1 with the
    quaternion Householder matrix H = I - 2 w w^H / (w^H w), w = x - alpha e_1,
    alpha = -(x_1 / |x_1|) ||x||.  With that alpha the scalar w^H x is real, so H x = alpha e_1.
    Afterwards a diagonal of unit quaternions D = diag(r_jj / |r_jj|) moves the phase of R's
    diagonal into Q:  Y = (Q D)(D^H R).
    """
    Y = np.asarray(Y, dtype=np.float64)
    _, m, n = Y.shape
    if m < n:
        raise ValueError("householder_qr needs rows >= cols")
    R = Y.copy()
    reflectors = []
    for j in range(n):
        x = R[:, j:, j]                                   # (4, m-j)
        nx = float(np.sqrt(np.sum(x * x)))
        if nx == 0.0:
            reflectors.append(None)
            continue
        x1 = x[:, 0]
        a1 = float(qnorm(x1))
        phase = x1 / a1 if a1 > 0.0 else np.array([1.0, 0.0, 0.0, 0.0])
        alpha = -phase * nx
        w = x.copy()
        w[:, 0] -= alpha
        ww = float(np.sum(w * w))
        wc = w[:, :, None]                                # column vector (4, m-j, 1)
        s = qmatmul(qH(wc), R[:, j:, j:])                 # w^H R  (4, 1, n-j)
        R[:, j:, j:] -= (2.0 / ww) * qmatmul(wc, s)
        reflectors.append((j, wc, ww))
    # Q = H_1 H_2 ... H_n [I_n; 0]
    Q = np.zeros((4, m, n))
    Q[0, :n, :n] = np.eye(n)
    for item in reversed(reflectors):
        if item is None:
            continue
        j, wc, ww = item
        s = qmatmul(qH(wc), Q[:, j:, :])
        Q[:, j:, :] -= (2.0 / ww) * qmatmul(wc, s)
    R = R[:, :n, :n]
    for c in range(4):
        R[c] = np.triu(R[c])
    # phase normalisation so that diag(R) is real and non-negative
    d = R[:, np.arange(n), np.arange(n)]                  # (4, n)
    nd = qnorm(d)
    unit = np.where(nd > 0.0, d / np.where(nd > 0.0, nd, 1.0), np.array([1.0, 0, 0, 0])[:, None])
    R = qmul(qconj(unit)[:, :, None], R)                  # row j times conj(d_j)
    Q = qmul(Q, unit[:, None, :])                         # column j times d_j
    idx = np.arange(n)
    R[1:, idx, idx] = 0.0
    R[0, idx, idx] = nd
    return Q, R


def qr(Y: np.ndarray):
    """The "QR" step of Algorithms 1-4: thin Householder QR with real non-negative diag(R)."""
    return householder_qr(Y)
