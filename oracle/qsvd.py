"""QSVD through the complex adjoint matrix (Def. 1, eq. qsvd).  Test infrastructure only.

Write a quaternion matrix as X = Xa + Xb j with complex Xa = X0 + X1 i and Xb = X2 + X3 i.
Its complex adjoint is the 2m x 2n complex matrix

    chi(X) = [[ Xa,        Xb       ],
              [ -conj(Xb), conj(Xa) ]],

a ring homomorphism: chi(XY) = chi(X) chi(Y) and chi(X^H) = chi(X)^H.  Every singular value
of X appears twice among those of chi(X) (Zhang 1997, cited for Def. 1).  A complex vector
[u; w] of length 2n is the first column of chi(x) for the quaternion vector x with
xa = u and xb = -conj(w); any unit vector in the two-dimensional singular subspace of a
doubled singular value therefore maps to a right singular vector of X (unique up to a right
unit-quaternion factor).  Picking one vector per pair is not described in the paper; the
oracle takes candidates in descending order and keeps a candidate when it is not already in
the quaternion span of the vectors kept so far (quaternion Gram-Schmidt guard).
"""
from __future__ import annotations

import numpy as np

from .quaternion import qmatmul, qH, qmul, qconj


def complex_adjoint(X: np.ndarray) -> np.ndarray:
    """chi(X) as a complex128 array of shape (2m, 2n)."""
    Xa = X[0] + 1j * X[1]
    Xb = X[2] + 1j * X[3]
    top = np.concatenate([Xa, Xb], axis=1)
    bot = np.concatenate([-np.conj(Xb), np.conj(Xa)], axis=1)
    return np.concatenate([top, bot], axis=0)


def from_complex_adjoint_column(c: np.ndarray) -> np.ndarray:
    """Quaternion vector x (4, n) whose chi(x) has first column c = [u; w]: xa = u, xb = -conj(w)."""
    n = c.shape[0] // 2
    u, w = c[:n], c[n:]
    return np.stack([u.real, u.imag, -w.real, w.imag])


def _qdot(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """a^H b for quaternion column vectors a, b of shape (4, n): a quaternion (4,)."""
    return qmatmul(qH(a[:, :, None]), b[:, :, None])[:, 0, 0]


def qsvd(X: np.ndarray, rank: int | None = None):
    """Return (U, s, V) with X ~= U diag(s) V^H, s descending, U^H U = V^H V = I.

    Right singular vectors come from chi(X)'s right singular vectors (one per doubled value,
    with the Gram-Schmidt guard); left ones are u_i = X v_i / s_i for s_i > 0."""
    X = np.asarray(X, dtype=np.float64)
    _, m, n = X.shape
    r = min(m, n) if rank is None else rank
    C = complex_adjoint(X)
    _, sc, Vh = np.linalg.svd(C, full_matrices=False)
    Vc = np.conj(Vh.T)
    kept, svals = [], []
    for t in range(Vc.shape[1]):
        if len(kept) == r:
            break
        v = from_complex_adjoint_column(Vc[:, t])
        for _ in range(2):
            for q in kept:
                v = v - qmul(q, _qdot(q, v)[:, None])
        nv = float(np.sqrt(np.sum(v * v)))
        if nv > 0.5:
            kept.append(v / nv)
            svals.append(sc[t])
    V = np.stack(kept, axis=2) if kept else np.zeros((4, n, 0))
    s = np.array(svals)
    XV = qmatmul(X, V)
    U = np.zeros((4, m, V.shape[2]))
    for i in range(V.shape[2]):
        if s[i] > 0.0:
            U[:, :, i] = XV[:, :, i] / s[i]
    # rank-deficient tail (s_i == 0): complete U from chi(X)'s left vectors with the same guard
    if np.any(s == 0.0):
        Uc, _, _ = np.linalg.svd(C, full_matrices=False)
        keptU = [U[:, :, i] for i in range(V.shape[2]) if s[i] > 0.0]
        for i in range(V.shape[2]):
            if s[i] > 0.0:
                continue
            for t in range(Uc.shape[1]):
                u = from_complex_adjoint_column(Uc[:, t])
                for _ in range(2):
                    for q in keptU:
                        u = u - qmul(q, _qdot(q, u)[:, None])
                nu = float(np.sqrt(np.sum(u * u)))
                if nu > 0.5:
                    U[:, :, i] = u / nu
                    keptU.append(U[:, :, i])
                    break
    return U, s, V


def tsvd(R: np.ndarray, k: int):
    """Truncated SVD (R, k): (L, s, Rt) with R ~= L diag(s) Rt^H keeping the k largest values.

    Algorithms 1, 2 and 4 name the factors by their role: for even v, Algorithm 2 writes
    [V_hat, S, U_hat] = TSVD(R^(2), k), i.e. L = V_hat and Rt = U_hat."""
    U, s, V = qsvd(R, rank=k)
    return U[:, :, :k], s[:k], V[:, :, :k]


def singular_values(X: np.ndarray) -> np.ndarray:
    """Quaternion singular values (descending): every other singular value of chi(X)."""
    sc = np.linalg.svd(complex_adjoint(np.asarray(X, dtype=np.float64)), compute_uv=False)
    return sc[0::2].copy()


def real_representation(X: np.ndarray) -> np.ndarray:
    """The 4m x 4n real matrix of left multiplication by X on R^4 coordinates.  Every singular
    value of X appears four times among its singular values (an independent check of chi)."""
    X0, X1, X2, X3 = X
    return np.block([
        [X0, -X1, -X2, -X3],
        [X1, X0, -X3, X2],
        [X2, X3, X0, -X1],
        [X3, -X2, X1, X0],
    ])
