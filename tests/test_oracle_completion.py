"""Pins for the oracle's quaternion matrix completion (Section 7, eqs. Step1 and Step2).

- eq. Step2 entry by entry: an observed entry takes M's value, an unobserved one X's.
- With every entry observed, C = M whatever the low-rank operator returns.
- With the exact truncated QSVD as the low-rank operator, the alternating updates are
  alternating projections onto the rank-k matrices and onto the matrices that agree with M on
  the sampling set, so the objective ||X - C||_F of eq. (MinRankCompl3) never increases.
- A matrix of exact rank k, sampled on 60 % of its entries, is recovered on the unobserved
  entries (both with the exact truncated QSVD and with Algorithm 2, which is exact on rank-k
  input, Section 3).
- M of exact rank k is a fixed point of one update.
"""
import numpy as np

import synth
from oracle import completion as oc
from oracle.qsvd import qsvd


def _exact_lowrank(k):
    def L(C):
        U, s, V = qsvd(C, rank=k)
        return U[:, :, :k], s[:k], V[:, :, :k]
    return L


def test_masked_update_entry_by_entry():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((4, 7, 5))
    X = rng.standard_normal((4, 7, 5))
    mask = (rng.random((7, 5)) < 0.5).astype(np.uint8)
    C = oc.masked_update(M, mask, X)
    for i in range(7):
        for j in range(5):
            want = M[:, i, j] if mask[i, j] else X[:, i, j]
            assert np.array_equal(C[:, i, j], want)
    C0 = oc.masked_update(M, mask, None)
    assert np.array_equal(C0[:, mask == 0], np.zeros((4, int((mask == 0).sum()))))
    assert np.array_equal(C0[:, mask == 1], M[:, mask == 1])


def test_full_mask_returns_the_observed_matrix():
    P = synth.completion_problem(30, 24, 4, missing=0.0, seed=3, noise=0.1)
    assert P.extra["mask"].all()
    C, U, S, V, _ = oc.complete(P.A, P.extra["mask"], 4, 3, 2, 2, P.Omega[:, :, :7])
    assert np.array_equal(C, P.A)


def test_objective_non_increasing_with_exact_lowrank():
    P = synth.completion_problem(40, 30, 3, missing=0.5, seed=5, noise=0.05)
    _, _, _, _, hist = oc.complete(P.A, P.extra["mask"], 3, 0, 2, 25, lowrank=_exact_lowrank(3))
    h = np.array(hist)
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-12) + 1e-13)
    assert h[-1] < 0.5 * h[0]


def test_recovery_of_exact_low_rank_matrix():
    P = synth.completion_problem(40, 30, 3, missing=0.4, seed=6)
    mask = P.extra["mask"]
    miss = mask == 0
    ref = np.sqrt((P.A[:, miss] ** 2).sum())
    C, _, _, _, _ = oc.complete(P.A, mask, 3, 0, 2, 150, lowrank=_exact_lowrank(3))
    assert np.sqrt(((C - P.A)[:, miss] ** 2).sum()) < 1e-4 * ref
    C2, _, S2, _, _ = oc.complete(P.A, mask, 3, 3, 2, 150, P.Omega[:, :, :6])
    assert np.sqrt(((C2 - P.A)[:, miss] ** 2).sum()) < 1e-4 * ref
    assert len(S2) == 3


def test_rank_k_matrix_is_a_fixed_point():
    P = synth.completion_problem(36, 28, 4, missing=0.5, seed=8)
    X = oc.low_rank_product(*_exact_lowrank(4)(P.A))
    assert np.abs(X - P.A).max() < 1e-12 * np.abs(P.A).max()
    C = oc.masked_update(P.A, P.extra["mask"], X)
    assert np.abs(C - P.A).max() < 1e-12 * np.abs(P.A).max()
