"""Quaternion matrix completion by alternating updates (Section 7, eqs. Step1 and Step2), in
float64.  Test infrastructure only.

The observed matrix M (m x n quaternion) is known on a sampling set, given as a 0/1 mask of
shape (m, n).  Starting from C = P_Omega(M) (the unobserved entries zero: the paper does not
state the starting point), each iteration takes
    X = L(C)                                          (eq. Step1)
    C = mask .* M + (1 - mask) .* X                   (eq. Step2)
where L is a rank-k approximation.  By default L is Algorithm 2 or 4 of `oracle.algorithms`
(the paper uses Algorithm 2 with two passes); `lowrank` replaces it, e.g. by the exact truncated
QSVD for the pins.  The same test matrix Omega serves every iteration (the caller passes it).
The Gaussian smoothing the paper applies to images after each iteration is image
post-processing, not part of the completion operator, and is not modelled.
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import numpy as np

from .algorithms import run
from .quaternion import qmatmul, qH


def masked_update(M: np.ndarray, mask: np.ndarray, X: Optional[np.ndarray]) -> np.ndarray:
    """eq. Step2: mask .* M + (1 - mask) .* X, entrywise over all four planes; X = None means
    X = 0 (this gives the starting point P_Omega(M))."""
    w = np.asarray(mask, dtype=np.float64)[None, :, :]
    out = w * np.asarray(M, dtype=np.float64)
    if X is not None:
        out = out + (1.0 - w) * np.asarray(X, dtype=np.float64)
    return out


def low_rank_product(U: np.ndarray, S: np.ndarray, V: np.ndarray) -> np.ndarray:
    """X = U diag(S) V^H."""
    return qmatmul(U * np.asarray(S)[None, None, :], qH(V))


def complete(M: np.ndarray, mask: np.ndarray, k: int, p: int, v: int, iters: int, Omega=None,
             algo: str = "alg2", side: str = "X",
             lowrank: Optional[Callable[[np.ndarray], Tuple[np.ndarray, np.ndarray, np.ndarray]]] = None):
    """`iters` alternating updates from C = P_Omega(M).  Returns (C, U, S, V, history) where C is
    the last eq. Step2 result, (U, S, V) the factors of the last X and history[t] the objective
    ||X^(t) - C^(t)||_F of eq. (MinRankCompl3) at iteration t."""
    C = masked_update(M, mask, None)
    U = S = V = None
    history = []
    for _ in range(iters):
        if lowrank is None:
            res = run(algo, C, k, p, v, Omega, side=side)
            U, S, V = res.U, res.S, res.V
        else:
            U, S, V = lowrank(C)
        X = low_rank_product(U, S, V)
        history.append(float(np.sqrt(((X - C) ** 2).sum())))
        C = masked_update(M, mask, X)
    return C, U, S, V, history
