"""Algorithms 1-4 of the paper, step by step, in float64.  Test infrastructure only.

Each function follows its algorithm's steps in the paper's order and notation: X is the
data matrix (I1 x I2), Omega the quaternion Gaussian test matrix of size I2 x (k+p) (passed
in, never drawn here), "QR" is `oracle.qr.qr` and "Truncated SVD" is `oracle.qsvd.tsvd`.
A pass (view) is one product with X or X^H; every function counts its passes and the number
of columns it multiplies X or X^H with, for the execution-cost statements of Section 6.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .quaternion import qmatmul, qH, qhstack
from .qr import qr
from .qsvd import tsvd, qsvd


@dataclass
class Result:
    U: np.ndarray
    S: np.ndarray
    V: np.ndarray
    Q1: Optional[np.ndarray] = None
    Q2: Optional[np.ndarray] = None
    R: Optional[np.ndarray] = None
    passes: int = 0
    columns: int = 0                   # sum over passes of the columns multiplied
    side: str = "X"                    # "X" or "XH" (Section 6)
    trace: List[str] = field(default_factory=list)


class _Counter:
    def __init__(self, X):
        self.X = X
        self.XH = qH(X)
        self.passes = 0
        self.columns = 0
        self.trace: List[str] = []

    def times(self, B):               # X B
        self.passes += 1
        self.columns += B.shape[2]
        self.trace.append("X")
        return qmatmul(self.X, B)

    def h_times(self, B):             # X^H B
        self.passes += 1
        self.columns += B.shape[2]
        self.trace.append("XH")
        return qmatmul(self.XH, B)


def alg1_classical(X, k: int, p: int, q: int, Omega) -> Result:
    """Algorithm 1: classical randomized subspace method, 2q+2 passes."""
    ops = _Counter(np.asarray(X, dtype=np.float64))
    Q1, _ = qr(ops.times(Omega))                       # [Q1, ~] = QR(X Omega)
    for _ in range(q):
        Q2, _ = qr(ops.h_times(Q1))                    # [Q2, ~] = QR(X^H Q1)
        Q1, _ = qr(ops.times(Q2))                      # [Q1, ~] = QR(X Q2)
    Q2, R = qr(ops.h_times(Q1))                        # [Q2, R] = QR(X^H Q1)
    Vh, S, Uh = tsvd(R, k)                             # [V_hat, S, U_hat] = TSVD(R, k)
    V = qmatmul(Q2, Vh)
    U = qmatmul(Q1, Uh)
    return Result(U, S, V, Q1, Q2, R, ops.passes, ops.columns, "X", ops.trace)


def alg2_arbitrary_pass(X, k: int, p: int, v: int, Omega) -> Result:
    """Algorithm 2: randomized truncated SVD with an arbitrary number v >= 2 of passes."""
    if v < 2:
        raise ValueError("Algorithm 2 needs v >= 2 passes")
    ops = _Counter(np.asarray(X, dtype=np.float64))
    Q2 = Omega                                         # Q2 is the Gaussian test matrix
    Q1 = R1 = R2 = None
    for i in range(1, v + 1):
        if i % 2 == 1:
            Q1, R1 = qr(ops.times(Q2))                 # [Q1, R1] = QR(X Q2)
        else:
            Q2, R2 = qr(ops.h_times(Q1))               # [Q2, R2] = QR(X^H Q1)
    if v % 2 == 0:
        Vh, S, Uh = tsvd(R2, k)                        # [V_hat, S, U_hat] = TSVD(R2, k)
        R = R2
    else:
        Uh, S, Vh = tsvd(R1, k)                        # [U_hat, S, V_hat] = TSVD(R1, k)
        R = R1
    V = qmatmul(Q2, Vh)
    U = qmatmul(Q1, Uh)
    return Result(U, S, V, Q1, Q2, R, ops.passes, ops.columns, "X", ops.trace)


def alg3_block_classical(X, k: int, p: int, q: int, Omega) -> Result:
    """Algorithm 3: classical block randomized subspace method, 2(q+1) passes."""
    ops = _Counter(np.asarray(X, dtype=np.float64))
    K = [ops.times(Omega)]                             # K0 = X Omega
    for _ in range(q):
        K.append(ops.times(ops.h_times(K[-1])))        # Ki = (X X^H) K_{i-1}
    Q, _ = qr(qhstack(K))                              # [Q, ~] = QR([K0 ... Kq])
    Yt = qH(ops.h_times(Q))                            # Y~ = Q^H X = (X^H Q)^H
    Uy, S, Vy = qsvd(Yt)                               # full SVD of Y~
    Uhat = qmatmul(Q, Uy)
    return Result(Uhat[:, :, :k], S[:k], Vy[:, :, :k], Q, None, None, ops.passes, ops.columns,
                  "X", ops.trace)


def alg4_block_flexible(X, k: int, p: int, v: int, Omega) -> Result:
    """Algorithm 4: flexible block Krylov with an arbitrary number v >= 2 of views."""
    if v < 2:
        raise ValueError("Algorithm 4 needs v >= 2 views")
    ops = _Counter(np.asarray(X, dtype=np.float64))
    Q2_blocks = {0: Omega}                             # Q2_0 = Omega
    Q1_blocks = {}
    s = (v - 1) // 2
    for j in range(1, s + 1):
        if 2 * j - 1 < v:
            Q1_blocks[j], _ = qr(ops.times(Q2_blocks[j - 1]))      # odd view: range side
        if 2 * j < v:
            Q2_blocks[j], _ = qr(ops.h_times(Q1_blocks[j]))
    if v % 2 == 0:
        Q1_blocks[s + 1], _ = qr(ops.times(Q2_blocks[s]))
        K1 = qhstack([Q1_blocks[j] for j in range(1, v // 2 + 1)])
        Q1, _ = qr(K1)
        Q2, R2 = qr(ops.h_times(Q1))
        Vh, S, Uh = tsvd(R2, k)
        R = R2
    else:
        K2 = qhstack([Q2_blocks[j] for j in range(1, (v - 1) // 2 + 1)])
        Q2, _ = qr(K2)
        Q1, R1 = qr(ops.times(Q2))
        Uh, S, Vh = tsvd(R1, k)
        R = R1
    V = qmatmul(Q2, Vh)
    U = qmatmul(Q1, Uh)
    return Result(U, S, V, Q1, Q2, R, ops.passes, ops.columns, "X", ops.trace)


def default_side(m: int, n: int, v: int) -> str:
    """Section 6: for even v prefer X^H when X has more columns than rows, else X; for odd v
    apply to X (the left factor is then the more accurate one, eq. mn12)."""
    if v % 2 == 0 and n > m:
        return "XH"
    return "X"


def run(algo: str, X, k: int, p: int, v: int, Omega, side: str = "X") -> Result:
    """Run Algorithm 2 ("alg2") or 4 ("alg4") on X or on X^H (Section 6).

    Applied to X^H the algorithm returns X^H ~= U' S V'^H, hence X ~= V' S U'^H; Omega must
    then have I1 rows."""
    f = {"alg2": alg2_arbitrary_pass, "alg4": alg4_block_flexible}[algo]
    if side == "X":
        return f(X, k, p, v, Omega)
    res = f(qH(np.asarray(X, dtype=np.float64)), k, p, v, Omega)
    return Result(res.V, res.S, res.U, res.Q2, res.Q1, res.R, res.passes, res.columns, "XH",
                  res.trace)
