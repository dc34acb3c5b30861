"""The allocation-free sketch entry point, qlr_qsketch_noalloc.

It exists for callers that cannot allocate device memory: a latency-critical serving loop keeps
cudaMalloc (which may synchronise the device and takes a driver-wide lock) out of its steady
state, and some host applications give all device memory to their own pool allocator.  The entry
point takes its scratch from one fixed device array in the library instead.

Checked here, through the C ABI: its product equals the FP64 oracle's Hamilton product (eq. 1
summed over the inner index) element by element within the tensor-core bound, and the context
entry point qlr_qsketch's product within twice that bound, on two calls in a row (the shared
array keeps the first call's contents, which must not leak into the second);
repeated calls allocate no device memory; sizes beyond the array give QLR_ENOMEM; degenerate
sizes behave as in qlr_qsketch.  The file name sorts after the other GPU test files."""
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
                                          ("TF32", "N", 300, 264, 5), ("TF32X3", "N", 4096, 4096, 110)])
def test_noalloc_matches_oracle_product(mode, op, m, n, l):
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    A = synth.gaussian_qmat(41 + m, m, n)
    rows_in = n if op == "N" else m
    rows_out = m if op == "N" else n
    Ad = dev_rowmajor(A, "bf16" if mode == "BF16" else "f32")
    Xd = dev_thin(synth.gaussian_qmat(42 + l, rows_in, l), "f32")
    o = qlr.OP_N if op == "N" else qlr.OP_H
    compute = getattr(qlr, "COMPUTE_" + mode)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    # the oracle product of the values the kernel consumes (A as stored, X rounded to BF16 in BF16 mode)
    Ah = host(Ad)
    Aop = Ah if op == "N" else Q.qH(Ah)
    Xh = host(Xd.to(torch.bfloat16)) if mode == "BF16" else host(Xd)
    want = Q.qmatmul(Aop, Xh)
    bound = 2 * _tol(mode, rows_in) * (Q.qnorm(Aop) @ Q.qnorm(Xh)) + 1e-30
    ctx = qlr.Context()
    Yctx = qlr.empty_thin(rows_out, l)
    qlr.qsketch(ctx, o, Ad, Xd, Yctx, compute)
    torch.cuda.synchronize()
    ref = host(Yctx)
    assert np.all(Q.qnorm(ref - want) <= bound)
    for call in range(2):
        Y = qlr.empty_thin(rows_out, l)
        Y.fill_(float("nan"))
        qlr.qsketch_noalloc(o, Ad, Xd, Y, compute, err=err)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        diff = Q.qnorm(host(Y) - want)
        assert np.all(np.isfinite(diff)), f"call {call}"
        assert np.all(diff <= bound), f"call {call}: {float((diff / bound).max())}"
        assert np.all(Q.qnorm(host(Y) - ref) <= 2 * bound), f"call {call} against qlr_qsketch"
    ctx.close()


def test_noalloc_allocates_no_device_memory():
    """After a first call (which loads the kernels and looks up the array's address), further
    calls leave the device's free memory unchanged: nothing is allocated per call."""
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    Ad = dev_rowmajor(synth.gaussian_qmat(7, 2048, 1536), "f32")
    Xd = dev_thin(synth.gaussian_qmat(8, 1536, 64), "f32")
    Xh = dev_thin(synth.gaussian_qmat(9, 2048, 64), "f32")
    Y, Z = qlr.empty_thin(2048, 64), qlr.empty_thin(1536, 64)
    qlr.qsketch_noalloc(qlr.OP_N, Ad, Xd, Y, qlr.COMPUTE_TF32X3)
    qlr.qsketch_noalloc(qlr.OP_H, Ad, Xh, Z, qlr.COMPUTE_TF32X3)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        qlr.qsketch_noalloc(qlr.OP_N, Ad, Xd, Y, qlr.COMPUTE_TF32X3)
        qlr.qsketch_noalloc(qlr.OP_H, Ad, Xh, Z, qlr.COMPUTE_TF32X3)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_degenerate_sizes():
    """An empty Y launches nothing; an empty inner dimension is an empty sum, Y = 0 (as qlr_qsketch)."""
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    for op in (qlr.OP_N, qlr.OP_H):
        A = torch.zeros(4, 0, 6, device="cuda") if op == qlr.OP_N else torch.zeros(4, 6, 0, device="cuda")
        qlr.qsketch_noalloc(op, A, qlr.empty_thin(6, 3), qlr.empty_thin(0, 3), qlr.COMPUTE_TF32X3)
        A = torch.ones(4, 5, 6, device="cuda")
        X = qlr.empty_thin(6 if op == qlr.OP_N else 5, 0)
        qlr.qsketch_noalloc(op, A, X, qlr.empty_thin(5 if op == qlr.OP_N else 6, 0), qlr.COMPUTE_TF32X3)
        A = torch.zeros(4, 5, 0, device="cuda") if op == qlr.OP_N else torch.zeros(4, 0, 5, device="cuda")
        Y = qlr.empty_thin(5, 3)
        Y.fill_(float("nan"))
        qlr.qsketch_noalloc(op, A, qlr.empty_thin(0, 3), Y, qlr.COMPUTE_TF32X3)
        torch.cuda.synchronize()
        assert bool(torch.all(Y == 0))


def test_noalloc_rejects_oversized_operands():
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    A = torch.zeros(4, 64, 200000, device="cuda")        # staged X would need > 128 MiB
    X = qlr.empty_thin(200000, 64)
    Y = qlr.empty_thin(64, 64)
    with pytest.raises(qlr.QlrError) as e:
        qlr.qsketch_noalloc(qlr.OP_N, A, X, Y, qlr.COMPUTE_TF32X3)
    assert e.value.code == qlr.ENOMEM
