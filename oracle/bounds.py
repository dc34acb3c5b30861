"""Expected-error bounds of Sections 4 and 5.  Test infrastructure only.

All bounds share the form  ( a * s_{k+1}^e + b * (sum_{j>k} s_j^{2e})^{1/2} )^{1/e}  with
a = 1 + 3 sqrt(k / (4p+2)) and b = 3 e sqrt(4k+4p+2) / (2p+2) (e = Euler's number), for an
exponent e that depends on the algorithm and the number of passes.
"""
from __future__ import annotations

import math

import numpy as np


def _coeffs(k: int, p: int):
    a = 1.0 + 3.0 * math.sqrt(k / (4.0 * p + 2.0))
    b = 3.0 * math.e * math.sqrt(4.0 * k + 4.0 * p + 2.0) / (2.0 * p + 2.0)
    return a, b


def power_bound(sigma: np.ndarray, k: int, p: int, expo: float) -> float:
    """(a sigma_{k+1}^expo + b (sum_{j>k} sigma_j^{2 expo})^{1/2})^{1/expo}; sigma descending,
    0-based array, so sigma_{k+1} is sigma[k]."""
    a, b = _coeffs(k, p)
    tail = np.asarray(sigma, dtype=np.float64)[k:]
    val = a * tail[0] ** expo + b * math.sqrt(float(np.sum(tail ** (2.0 * expo))))
    return val ** (1.0 / expo)


def lemma1(sigma, k: int, p: int, q: int = 0) -> float:
    """Lemma 1: E||X_hat^(q) - X||_2 for Algorithm 1 with q power iterations (exponent 2q+1)."""
    return power_bound(sigma, k, p, 2 * q + 1)


def theorem3(sigma, k: int, p: int, q: int) -> float:
    """Theorem 3: E||X - X Q2 Q2^H||_2 with exponent 2q."""
    return power_bound(sigma, k, p, 2 * q)


def mn11_12(sigma, k: int, p: int, v: int):
    """eqs. (mn11) / (mn12): bounds on (||X - Q1 Q1^H X||, ||X - X Q2 Q2^H||) after v passes of
    Algorithm 2.  Even v: exponents (v-1, v); odd v: exponents (v, v-1)."""
    if v % 2 == 0:
        return power_bound(sigma, k, p, v - 1), power_bound(sigma, k, p, v)
    return power_bound(sigma, k, p, v), power_bound(sigma, k, p, v - 1)


def lemma4(sigma, k: int, p: int, q: int) -> float:
    """Lemma 4 (eq. BK-safe): block Krylov range error with exponent 2q+1."""
    return power_bound(sigma, k, p, 2 * q + 1)


def corollary5(sigma, k: int, p: int) -> float:
    """Corollary 5: the q = 0 case of Lemma 4."""
    return power_bound(sigma, k, p, 1)


def theorem6(sigma, k: int, p: int, v: int) -> float:
    """Theorem 6: flexible block Krylov with v views, exponent alpha_v = v - 1 (range error for
    even v, co-range error for odd v)."""
    return power_bound(sigma, k, p, v - 1)
