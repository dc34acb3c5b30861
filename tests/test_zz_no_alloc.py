"""The allocation-free sketch entry point (qlr_qsketch_noalloc) gives the same product as the
context-based qlr_qsketch, for callers that must not call cudaMalloc (latency-critical loops,
hosts whose pool allocator owns all device memory).  Two calls in a row check that the shared
scratch array's leftover contents from one call do not leak into the next.  This file is named
to be collected last."""
import numpy as np
import pytest
import torch

import synth
from oracle import quaternion as Q
from tests._qutil import dev_rowmajor, dev_thin, host

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _tol(mode, K):
    acc = 4.0 * K * U32
    return {"BF16": acc, "TF32": 2.0 ** -9 + acc, "TF32X3": 2.0 ** -19 + acc}[mode]


@pytest.mark.parametrize("mode,op,m,n,l", [("TF32X3", "N", 1024, 768, 37), ("TF32X3", "H", 1024, 768, 37),
                                          ("BF16", "N", 640, 2048, 110), ("BF16", "H", 640, 2048, 110),
                                          ("TF32", "N", 300, 264, 5)])
def test_noalloc_matches_context_entry_point(mode, op, m, n, l):
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    ctx = qlr.Context(0)
    A = synth.gaussian_qmat(41 + m, m, n)
    rows_in = n if op == "N" else m
    rows_out = m if op == "N" else n
    Ad = dev_rowmajor(A, "bf16" if mode == "BF16" else "f32")
    Xd = dev_thin(synth.gaussian_qmat(42 + l, rows_in, l), "f32")
    o = qlr.OP_N if op == "N" else qlr.OP_H
    compute = getattr(qlr, "COMPUTE_" + mode)
    Yref = qlr.empty_thin(rows_out, l)
    qlr.qsketch(ctx, o, Ad, Xd, Yref, compute)
    assert ctx.sync() == 0
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    Ah = host(Ad)
    Aop = Ah if op == "N" else Q.qH(Ah)
    Xh = host(Xd.to(torch.bfloat16)) if mode == "BF16" else host(Xd)
    bound = 2 * _tol(mode, rows_in) * (Q.qnorm(Aop) @ Q.qnorm(Xh)) + 1e-30
    for call in range(2):
        Y = qlr.empty_thin(rows_out, l)
        Y.fill_(float("nan"))
        qlr.qsketch_noalloc(o, Ad, Xd, Y, compute, err=err)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        diff = Q.qnorm(host(Y) - host(Yref))
        assert np.all(np.isfinite(diff)), f"call {call}"
        assert np.all(diff <= bound), f"call {call}: {float((diff / bound).max())}"
    ctx.close()


def test_noalloc_rejects_oversized_operands():
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    A = torch.zeros(4, 64, 200000, device="cuda")        # staged X would need > 32 MiB
    X = qlr.empty_thin(200000, 64)
    Y = qlr.empty_thin(64, 64)
    with pytest.raises(qlr.QlrError) as e:
        qlr.qsketch_noalloc(qlr.OP_N, A, X, Y, qlr.COMPUTE_TF32X3)
    assert e.value.code == qlr.ENOMEM
