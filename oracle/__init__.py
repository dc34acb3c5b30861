"""FP64 CPU oracle for the pass-efficient randomized quaternion low-rank approximation.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
baseline leg import this package.  The GPU library never calls it and shares no code with it.

The oracle is plain, slow and written to be checked against the paper by eye:

* ``quaternion``  -- quaternion numbers and matrices stored as four real planes; the Hamilton
                    product (Section 2, eq. 1), conjugate, norm, inverse, X^H (Section 2).
* ``qr``          -- thin quaternion QR (Def. 1, eq. QQR) by Householder reflections, with the
                    diagonal of R normalised to be real and positive.
* ``qsvd``        -- QSVD (Def. 1, eq. qsvd) through the complex adjoint matrix and LAPACK, and
                    the truncated SVD the algorithms call.
* ``algorithms``  -- Algorithms 1, 2, 3 and 4 step by step, plus the X / X^H side choice of
                    Section 6.
* ``norms``       -- spectral norms of quaternion matrices and of the projection residuals the
                    theorems bound.
* ``bounds``      -- the expected-error bounds of Lemma 1, Theorem 3 (eqs. mn11/mn12),
                    Lemma 4 / Corollary 5 and Theorem 6.
* ``completion``  -- quaternion matrix completion by the alternating updates of Section 7
                    (eqs. Step1 and Step2) around a rank-k approximation.

Every floating-point step runs in float64.  Where a function is only checked against itself
it says "parity unpinned" in its docstring; all functions here are pinned by the tests in
``tests/test_oracle_*.py``.
"""
from . import quaternion, qr, qsvd, algorithms, norms, bounds, completion  # noqa: F401
