"""Failure detection without a GPU fault: a bounded device wait that nothing satisfies gives up
after its limit, the context's device error word reports QLR_ETIMEOUT exactly once, and the
context keeps running work afterwards (a small FP64 sketch checked against the oracle)."""
import time

import numpy as np
import pytest
import torch

from oracle import quaternion as Q
from tests._qutil import dev_rowmajor, dev_thin, host

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    ctx = qlr.Context(0)
    t0 = time.perf_counter()
    qlr.selftest_wait_timeout(ctx)
    assert ctx.sync() == qlr.ETIMEOUT
    assert time.perf_counter() - t0 > 1.0          # the wait ran to its limit
    assert ctx.sync() == 0                         # reported once, then cleared
    rng = np.random.default_rng(3)
    A = rng.standard_normal((4, 40, 30))
    X = rng.standard_normal((4, 30, 7))
    Y = qlr.empty_thin(40, 7, torch.float64)
    qlr.qsketch(ctx, qlr.OP_N, dev_rowmajor(A, "f64"), dev_thin(X, "f64"), Y, qlr.COMPUTE_F64)
    assert ctx.sync() == 0
    np.testing.assert_allclose(host(Y), Q.qmatmul(A, X), rtol=0, atol=1e-12 * np.abs(A).max() * 30)
    ctx.close()
