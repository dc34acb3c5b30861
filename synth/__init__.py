"""Seeded synthetic inputs shared by the FP64 oracle, the GPU tests and the benchmark.

This module only builds inputs: quaternion test matrices with a prescribed spectrum or
structure, and the Gaussian test matrix Omega that both paths receive.  It implements none
of the low-rank method (no sketch products, no QR of a sketch, no truncated SVD).  Building a
matrix with prescribed singular values needs a few quaternion products and reflectors; those
are private helpers here, written for input construction only.

Storage convention: a quaternion matrix is a float64 ndarray of shape (4, rows, cols); the
leading axis holds the planes (real, i, j, k) in that order (the paper's X1..X4, Section 2).

Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; constants as published by Vigna) used counter-style, i.e. draw
number t of a stream is the SplitMix64 output for state seed + (t+1)*0x9E3779B97F4A7C15.
Uniforms take the top 53 bits; normals use the Box-Muller transform on consecutive pairs.
A quaternion Gaussian matrix (Def. 2) is filled plane-major, column-major:
element (c, i, j) of an r x s matrix is normal number c*r*s + j*r + i of its stream.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

# stream tags (one independent stream per use)
TAG_LEFT, TAG_RIGHT, TAG_PHASE_U, TAG_PHASE_V, TAG_NOISE, TAG_OMEGA, TAG_SIZES, TAG_FIELD, TAG_MASK = range(1, 10)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output number `counter` (0-based) of the generator seeded with `seed`."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        return _mix(z)


def stream_seed(seed: int, *tags: int) -> int:
    """Derive an independent stream seed from a base seed and a tuple of small tags."""
    s = seed & 0xFFFFFFFFFFFFFFFF
    for t in tags:
        s = int(splitmix64(s, np.array([t], dtype=np.uint64))[0])
    return s


def uniform(seed: int, count: int) -> np.ndarray:
    """`count` uniforms in [0, 1) (top 53 bits of each SplitMix64 output)."""
    out = np.empty(count, dtype=np.float64)
    for lo in range(0, count, _CHUNK):
        hi = min(count, lo + _CHUNK)
        z = splitmix64(seed, np.arange(lo, hi, dtype=np.uint64))
        out[lo:hi] = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return out


def gaussian(seed: int, count: int) -> np.ndarray:
    """`count` iid N(0,1) numbers by Box-Muller on consecutive uniform pairs."""
    npair = (count + 1) // 2
    out = np.empty(2 * npair, dtype=np.float64)
    for lo in range(0, npair, _CHUNK):
        hi = min(npair, lo + _CHUNK)
        idx = np.arange(2 * lo, 2 * hi, dtype=np.uint64)
        z = splitmix64(seed, idx)
        u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        u1 = 1.0 - u[0::2]          # (0, 1]
        u2 = u[1::2]
        r = np.sqrt(-2.0 * np.log(u1))
        out[2 * lo:2 * hi:2] = r * np.cos(2.0 * np.pi * u2)
        out[2 * lo + 1:2 * hi:2] = r * np.sin(2.0 * np.pi * u2)
    return out[:count]


def gaussian_qmat(seed: int, rows: int, cols: int, real_only: bool = False) -> np.ndarray:
    """Gaussian quaternion matrix (Def. 2): four iid N(0,1) planes, plane-major column-major fill.

    With real_only=True only plane 0 is drawn (the real-Gaussian test matrix the experiments
    of Section 8 use); the other planes are zero.
    """
    nplanes = 1 if real_only else 4
    g = gaussian(seed, nplanes * rows * cols).reshape(nplanes, cols, rows).transpose(0, 2, 1)
    out = np.zeros((4, rows, cols), dtype=np.float64)
    out[:nplanes] = g
    return out


# ---------------------------------------------------------------------------------------
# private quaternion helpers (input construction only)
# Hamilton product sign table: (pq)_d = sum_c SGN[c][d] * p_c * q_{c xor d}
_SGN = np.array([[1, 1, 1, 1], [-1, 1, -1, 1], [-1, 1, 1, -1], [-1, -1, 1, 1]], dtype=np.float64)
_CONJ = np.array([1.0, -1.0, -1.0, -1.0])


def _qmm(P: np.ndarray, Q: np.ndarray) -> np.ndarray:
    out = np.zeros((4, P.shape[1], Q.shape[2]), dtype=np.float64)
    for c in range(4):
        for d in range(4):
            out[d] += _SGN[c, d] * (P[c] @ Q[c ^ d])
    return out


def _unit_quaternions(seed: int, count: int) -> np.ndarray:
    g = gaussian(seed, 4 * count).reshape(4, count)
    return g / np.sqrt((g * g).sum(axis=0, keepdims=True))


def _reflect_left(M: np.ndarray, w: np.ndarray) -> None:
    """M <- (I - 2 w w^H / |w|^2) M in place; w has shape (4, m)."""
    ww = float((w * w).sum())
    # P[c][e] = w_e^T M_c ; s = w^H M = sum over c of conj(w)_e M_c with the Hamilton signs
    P = np.stack([w @ M[c] for c in range(4)])            # (4 c, 4 e, n)
    s = np.zeros((4, M.shape[2]))
    for e in range(4):
        for d in range(4):
            s[d] += _SGN[e, d] * _CONJ[e] * P[e ^ d, e]
    # M -= (2/ww) * w s   (column w times row s)
    for d in range(4):
        coef = np.stack([_SGN[c, d] * s[c ^ d] for c in range(4)])  # (4, n)
        M[d] -= (2.0 / ww) * (w.T @ coef)


def _reflect_right(M: np.ndarray, w: np.ndarray) -> None:
    """M <- M (I - 2 w w^H / |w|^2) in place; w has shape (4, n)."""
    ww = float((w * w).sum())
    # t = M w  (m-vector), then M -= (2/ww) t w^H
    t = np.zeros((4, M.shape[1]))
    for c in range(4):
        for d in range(4):
            t[d] += _SGN[c, d] * (M[c] @ w[c ^ d])
    wh = w * _CONJ[:, None]
    for d in range(4):
        coef = np.stack([_SGN[c, d] * wh[c ^ d] for c in range(4)])  # (4 c, n)
        M[d] -= (2.0 / ww) * (t.T @ coef)


def _orthonormal_columns(G: np.ndarray) -> np.ndarray:
    """Modified Gram-Schmidt, run twice, on the columns of a quaternion matrix (4, m, r)."""
    Q = G.copy()
    r = Q.shape[2]
    for _ in range(2):
        for j in range(r):
            v = Q[:, :, j:j + 1]
            for i in range(j):
                qi = Q[:, :, i:i + 1]
                h = _qmm(qi.transpose(0, 2, 1) * _CONJ[:, None, None], v)  # q_i^H v (1x1)
                v = v - _qmm(qi, h)
            v = v / math.sqrt(float((v * v).sum()))
            Q[:, :, j:j + 1] = v
    return Q


# ---------------------------------------------------------------------------------------
@dataclass
class Problem:
    """One low-rank problem: quaternion A (4, m, n), target rank k, oversampling p, passes v."""
    name: str
    A: np.ndarray
    k: int
    p: int
    v: int
    Omega: np.ndarray
    sigma: Optional[np.ndarray] = None     # constructed singular values (descending), if known
    pure: bool = False
    extra: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.A.shape[1]

    @property
    def n(self) -> int:
        return self.A.shape[2]

    @property
    def ell(self) -> int:
        return self.k + self.p


def spectrum_matrix(m: int, n: int, sigma: np.ndarray, seed: int, n_reflectors: int = 8) -> np.ndarray:
    """A = U diag(sigma) V^H with U, V 'Haar-like': a random unit-quaternion diagonal followed by
    `n_reflectors` random quaternion Householder reflectors on each side."""
    r = min(m, n)
    assert sigma.shape == (r,)
    du = _unit_quaternions(stream_seed(seed, TAG_PHASE_U), r)
    dv = _unit_quaternions(stream_seed(seed, TAG_PHASE_V), r)
    # diagonal entries du_i * sigma_i * conj(dv_i)
    diag = np.zeros((4, r))
    dvc = dv * _CONJ[:, None]
    for c in range(4):
        for d in range(4):
            diag[d] += _SGN[c, d] * du[c] * dvc[c ^ d]
    diag *= sigma[None, :]
    M = np.zeros((4, m, n), dtype=np.float64)
    idx = np.arange(r)
    M[:, idx, idx] = diag
    for t in range(n_reflectors):
        w = gaussian(stream_seed(seed, TAG_LEFT, t), 4 * m).reshape(4, m)
        _reflect_left(M, w)
    for t in range(n_reflectors):
        w = gaussian(stream_seed(seed, TAG_RIGHT, t), 4 * n).reshape(4, n)
        _reflect_right(M, w)
    return M


def omega_for(seed: int, rows: int, ell: int, real_only: bool = False) -> np.ndarray:
    return gaussian_qmat(stream_seed(seed, TAG_OMEGA), rows, ell, real_only=real_only)


def config1(seed: int = 1234) -> Problem:
    """Plain 2-pass randomized QSVD in FP64 on a 256 x 192 matrix A = U diag(sigma) V^H + noise.
    U, V: Gram-Schmidt orthonormalised Gaussian quaternion matrices; sigma_i = 0.5^i (i = 0..9);
    iid quaternion Gaussian noise scaled by 1e-6; k = 10, p = 5, v = 2."""
    m, n, r = 256, 192, 10
    sigma = 0.5 ** np.arange(r)
    U = _orthonormal_columns(gaussian_qmat(stream_seed(seed, TAG_LEFT), m, r))
    V = _orthonormal_columns(gaussian_qmat(stream_seed(seed, TAG_RIGHT), n, r))
    VH = V.transpose(0, 2, 1) * _CONJ[:, None, None]
    A = _qmm(U * sigma[None, None, :], VH)
    A += 1e-6 * gaussian_qmat(stream_seed(seed, TAG_NOISE), m, n)
    k, p = 10, 5
    return Problem("c1", A, k, p, 2, omega_for(seed, n, k + p), sigma=sigma)


def config_slow_decay(m: int = 4096, n: int = 4096, k: int = 100, p: int = 10, v: int = 4,
                      seed: int = 1235) -> Problem:
    """FP32 arbitrary-pass workload: sigma_i = 1/i with Haar-like singular vectors."""
    r = min(m, n)
    sigma = 1.0 / np.arange(1, r + 1)
    A = spectrum_matrix(m, n, sigma, seed)
    return Problem(f"slowdecay{m}x{n}", A, k, p, v, omega_for(seed, n, k + p), sigma=sigma)


def config2(v: int = 4) -> Problem:
    return config_slow_decay(4096, 4096, 100, 10, v, seed=1235)


def config_exp_decay(m: int = 16384, n: int = 8192, k: int = 200, p: int = 20, v: int = 4,
                     seed: int = 1236, rate: float = 50.0) -> Problem:
    """Mixed-precision workload: sigma_i = exp(-i/50), Haar-like singular vectors."""
    r = min(m, n)
    sigma = np.exp(-np.arange(1, r + 1) / rate)
    A = spectrum_matrix(m, n, sigma, seed)
    return Problem(f"expdecay{m}x{n}", A, k, p, v, omega_for(seed, n, k + p), sigma=sigma)


def config3() -> Problem:
    return config_exp_decay(16384, 8192, 200, 20, 4, seed=1236)


def colour_field(m: int, n: int, seed: int, terms: int = 64, fmax: int = 8, noise: float = 0.05) -> np.ndarray:
    """Pure quaternion image-like matrix: for each of the i, j, k planes, a sum of `terms` 2-D
    cosines a cos(2 pi (fx x / W + fy y / H) + phi) with fx, fy ~ U{0..fmax}, a ~ N(0,1),
    phi ~ U[0, 2 pi); min-max scaled to [0, 1]; plus U[-noise, noise] noise.  Rows index y
    (H = m), columns index x (W = n)."""
    A = np.zeros((4, m, n), dtype=np.float64)
    y = np.arange(m, dtype=np.float64)[:, None] / m
    x = np.arange(n, dtype=np.float64)[None, :] / n
    for c in (1, 2, 3):
        u = uniform(stream_seed(seed, TAG_FIELD, c), 3 * terms)
        fx = np.floor(u[:terms] * (fmax + 1))
        fy = np.floor(u[terms:2 * terms] * (fmax + 1))
        phi = 2.0 * np.pi * u[2 * terms:]
        a = gaussian(stream_seed(seed, TAG_FIELD, 10 + c), terms)
        # cos(b + c) = cos b cos c - sin b sin c with b = 2 pi fy y, c = 2 pi fx x + phi
        by = 2.0 * np.pi * y * fy[None, :]                     # (m, terms)
        cx = 2.0 * np.pi * fx[:, None] * x + phi[:, None]      # (terms, n)
        left = np.concatenate([np.cos(by) * a[None, :], -np.sin(by) * a[None, :]], axis=1)
        right = np.concatenate([np.cos(cx), np.sin(cx)], axis=0)
        F = left @ right
        lo, hi = F.min(), F.max()
        F = (F - lo) / (hi - lo) if hi > lo else np.zeros_like(F)
        F += noise * (2.0 * uniform(stream_seed(seed, TAG_NOISE, c), m * n).reshape(m, n) - 1.0)
        A[c] = F
    return A


def config_colour(m: int = 20000, n: int = 10000, k: int = 50, b: int = 60, v: int = 6,
                  seed: int = 1237) -> Problem:
    """Pass-efficient block Krylov workload on a pure quaternion image-like matrix; block size b."""
    A = colour_field(m, n, seed)
    return Problem(f"colour{m}x{n}", A, k, b - k, v, omega_for(seed, n, b), pure=True)


def config4() -> Problem:
    return config_colour(20000, 10000, 50, 60, 6, seed=1237)


def batched_problems(count: int = 512, seed: int = 1238, mmin: int = 64, mmax: int = 1024,
                     nmin: int = 64, nmax: int = 768, rmin: int = 8, rmax: int = 64,
                     p: int = 8, v: int = 3, noise: float = 1e-3) -> List[Problem]:
    """Many pure quaternion matrices of uneven sizes, each of exact rank r plus noise.

    m ~ U{mmin..mmax}, n ~ U{nmin..nmax}, r ~ U{rmin..rmax}; A = B C with B a real Gaussian
    m x r matrix and C a pure Gaussian quaternion r x n matrix (real times pure stays pure and
    has rank r), scaled to unit RMS real component over the i, j, k planes; then iid
    N(0, noise^2) on the i, j, k planes.  k = r and ell = min(r + p, m, n)."""
    u = uniform(stream_seed(seed, TAG_SIZES), 3 * count).reshape(3, count)
    ms = mmin + np.floor(u[0] * (mmax - mmin + 1)).astype(int)
    ns = nmin + np.floor(u[1] * (nmax - nmin + 1)).astype(int)
    rs = rmin + np.floor(u[2] * (rmax - rmin + 1)).astype(int)
    out = []
    for i in range(count):
        m, n, r = int(ms[i]), int(ns[i]), int(rs[i])
        s = stream_seed(seed, 100 + i)
        B = gaussian(stream_seed(s, TAG_LEFT), m * r).reshape(r, m).T
        C = gaussian(stream_seed(s, TAG_RIGHT), 3 * r * n).reshape(3, n, r).transpose(0, 2, 1)
        A = np.zeros((4, m, n))
        for c in range(3):
            A[c + 1] = B @ C[c]
        A /= math.sqrt(float((A[1:] ** 2).mean()))
        A[1:] += noise * gaussian(stream_seed(s, TAG_NOISE), 3 * m * n).reshape(3, n, m).transpose(0, 2, 1)
        ell = min(r + p, m, n)
        out.append(Problem(f"batch{i}", A, r, ell - r, v, omega_for(s, n, ell), pure=True,
                           extra={"rank": r}))
    return out


def completion_problem(m: int, n: int, rank: int, missing: float = 0.7, seed: int = 1239, noise: float = 0.0,
                       k: Optional[int] = None, p: int = 10, v: int = 2) -> Problem:
    """Matrix-completion input (Section 7): M, a pure quaternion matrix of exact rank `rank`
    (a real Gaussian m x rank matrix times a pure Gaussian quaternion rank x n matrix, scaled to
    unit RMS over the i, j, k planes) plus iid N(0, noise^2) on the i, j, k planes, and a 0/1
    observation mask (uint8, m x n, 1 = observed) that removes each entry independently with
    probability `missing` (a uniform below `missing` removes it).  Stands in for the paper's
    colour images with 70 % of the pixels removed uniformly at random (Section 8).  k defaults to
    `rank`; Omega is n x (k + p).  The mask is in extra["mask"]."""
    k = rank if k is None else k
    B = gaussian(stream_seed(seed, TAG_LEFT), m * rank).reshape(rank, m).T
    C = gaussian(stream_seed(seed, TAG_RIGHT), 3 * rank * n).reshape(3, n, rank).transpose(0, 2, 1)
    A = np.zeros((4, m, n))
    for c in range(3):
        A[c + 1] = B @ C[c]
    A /= math.sqrt(float((A[1:] ** 2).mean()))
    if noise > 0.0:
        A[1:] += noise * gaussian(stream_seed(seed, TAG_NOISE), 3 * m * n).reshape(3, n, m).transpose(0, 2, 1)
    u = uniform(stream_seed(seed, TAG_MASK), m * n).reshape(m, n)
    mask = (u >= missing).astype(np.uint8)
    return Problem(f"complete{m}x{n}r{rank}", A, k, p, v, omega_for(seed, n, k + p), pure=True,
                   extra={"mask": mask, "rank": rank, "missing": missing})


def random_lowrank_problem(m: int, n: int, rank: int = 50, seed: int = 1241, p: int = 10, v: int = 2) -> Problem:
    """The random low-rank example of the experiments (Section 8): A = B C with B (m x rank) and
    C (rank x n) Gaussian quaternion matrices (Def. 2), so A has rank `rank`; k = rank, Omega is
    n x (rank + p).  The paper runs m = n = 500, 1000, ..., 4000 with rank 50 and does not state p."""
    B = gaussian_qmat(stream_seed(seed, TAG_LEFT, m, n), m, rank)
    C = gaussian_qmat(stream_seed(seed, TAG_RIGHT, m, n), rank, n)
    A = _qmm(B, C)
    return Problem(f"randlr{m}x{n}r{rank}", A, rank, p, v, omega_for(stream_seed(seed, m, n), n, rank + p),
                   extra={"rank": rank})
