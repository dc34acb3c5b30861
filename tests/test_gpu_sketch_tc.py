"""Parity of the tcgen05 sketch products (BF16, TF32, rounded TF32, 3xTF32) against the FP64 oracle product of
the values the kernel consumes.  Element-wise bounds: |err_ij| <= tol * sum_k |a_ik| |x_kj|
with tol from the mode's input rounding plus FP32 accumulation."""
import numpy as np
import pytest
import torch

import synth
from oracle import quaternion as Q
from tests._qutil import dev_rowmajor, dev_thin, host

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    c = qlr.Context(0)
    yield c
    c.close()


def _bf16(x):
    return torch.from_numpy(x).float().to(torch.bfloat16).double().numpy()


def _tol(mode, K):
    acc = 4.0 * K * U32
    return {"BF16": acc, "TF32": 2.0 ** -9 + acc, "TF32_RN": 2.0 ** -10 + acc, "TF32X3": 2.0 ** -19 + acc}[mode]


SHAPES = [(256, 192, 15, False), (300, 264, 37, False), (129, 1000, 5, False), (1000, 128, 112, False),
          (77, 40, 128, True), (200, 120, 220, False), (513, 1024, 64, False), (16, 8, 1, False),
          (640, 2048, 110, True),
          # pure, l = 180: 3xTF32 op N runs the fused output planes over three 64-column blocks
          (300, 504, 180, True)]


@pytest.mark.parametrize("m,n,l,pure", SHAPES)
@pytest.mark.parametrize("mode", ["TF32X3", "BF16", "TF32", "TF32_RN"])
@pytest.mark.parametrize("op", ["N", "H"])
def test_sketch_tc_parity(ctx, m, n, l, pure, mode, op):
    from paper_2507_13731_gb300 import qlr
    A = synth.gaussian_qmat(31 + m + n, m, n)
    if pure:
        A[0] = 0.0
    rows_in = n if op == "N" else m
    X = synth.gaussian_qmat(32 + l, rows_in, l)
    Ad = dev_rowmajor(A, "bf16" if mode == "BF16" else "f32", pure=pure)
    Xd = dev_thin(X, "f32")
    Ah = host(Ad)
    Xh = _bf16(host(Xd)) if mode == "BF16" else host(Xd)
    rows_out = m if op == "N" else n
    Yd = qlr.empty_thin(rows_out, l)
    Yd.fill_(float("nan"))
    qlr.qsketch(ctx, qlr.OP_N if op == "N" else qlr.OP_H, Ad, Xd, Yd, getattr(qlr, "COMPUTE_" + mode))
    assert ctx.sync() == 0
    Aop = Ah if op == "N" else Q.qH(Ah)
    want = Q.qmatmul(Aop, Xh)
    bound = _tol(mode, rows_in) * (Q.qnorm(Aop) @ Q.qnorm(Xh)) + 1e-30
    err = Q.qnorm(host(Yd) - want)
    assert np.all(np.isfinite(err))
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("op", ["N", "H"])
def test_tf32x3_full_size_sampled(ctx, op):
    """Slow-decay 4096 x 4096 FP32 workload (l = 110) in the launch configuration the benchmark
    times: 64 sampled output rows against the oracle."""
    from paper_2507_13731_gb300 import qlr
    P = synth.config_slow_decay(4096, 4096, 100, 10, 4)
    Ad, Xd = dev_rowmajor(P.A, "f32"), dev_thin(P.Omega, "f32")
    Yd = qlr.empty_thin(4096, 110)
    o = qlr.OP_N if op == "N" else qlr.OP_H
    qlr.qsketch(ctx, o, Ad, Xd, Yd, qlr.COMPUTE_TF32X3)
    assert ctx.sync() == 0
    rows = np.random.default_rng(1).choice(4096, 64, replace=False)
    Ah, Xh = host(Ad), host(Xd)
    Aop = Ah[:, rows, :] if op == "N" else Q.qH(Ah)[:, rows, :]
    want = Q.qmatmul(Aop, Xh)
    bound = _tol("TF32X3", 4096) * (Q.qnorm(Aop) @ Q.qnorm(Xh))
    assert np.all(Q.qnorm(host(Yd)[:, rows, :] - want) <= bound)


def test_tc_unsupported_alignment_is_reported(ctx):
    from paper_2507_13731_gb300 import qlr
    A = torch.zeros(4, 10, 7, device="cuda")      # row pitch 28 B: not a multiple of 16
    X = qlr.empty_thin(7, 3)
    Y = qlr.empty_thin(10, 3)
    with pytest.raises(qlr.QlrError) as e:
        qlr.qsketch(ctx, qlr.OP_N, A, X, Y, qlr.COMPUTE_TF32X3)
    assert e.value.code == qlr.EUNSUPPORTED


@pytest.mark.parametrize("mode", ["TF32X3", "TF32_RN"])
@pytest.mark.parametrize("op", ["N", "H"])
def test_long_one_signed_reduction(ctx, op, mode):
    """3xTF32 on data of one sign with a long reduction (K = 20000) and one output tile per SM (no
    stream-K split): the tensor cores' FP32 accumulation does not round to nearest, so adding all
    7500 MMAs of an output's reduction into one accumulator drifts by ~0.5 ulp per addition (about
    3e-4 relative here, all of one sign); the kernel reduces in chunks of 32 stages added in
    round-to-nearest FP32, which keeps every sampled entry within 2.5e-5 of the FP64 oracle product
    relative to sum_k |a_ik| |x_kj|.  Rounded TF32 (one product) gets there too: its operands are
    rounded to nearest (zero-mean errors, ~5e-6 relative on this sum), where the tensor cores'
    own truncation would shrink every product by ~2^-12 (~3e-4 of the sum), and its chunks hold
    512 reduction elements."""
    from paper_2507_13731_gb300 import qlr
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    M, K, l = sms * 128, 20000, 64
    g = torch.Generator(device="cuda").manual_seed(11)
    A = torch.rand(3, M, K, device="cuda", generator=g) if op == "N" else \
        torch.rand(3, K, M, device="cuda", generator=g)             # pure, entries in [0, 1)
    X = qlr.to_thin(torch.rand(4, K, l, device="cuda", generator=g))
    Y = qlr.empty_thin(M, l)
    qlr.qsketch(ctx, qlr.OP_N if op == "N" else qlr.OP_H, A, X, Y, getattr(qlr, "COMPUTE_" + mode))
    assert ctx.sync() == 0
    rows = torch.from_numpy(np.random.default_rng(3).choice(M, 48, replace=False)).cuda()
    Ar = A[:, rows, :] if op == "N" else A[:, :, rows].transpose(1, 2)
    Ah = np.concatenate([np.zeros((1, 48, K)), Ar.double().cpu().numpy()])
    Aop = Ah if op == "N" else Q.qconj(Ah)
    Xh = host(X)
    want = Q.qmatmul(Aop, Xh)
    scale = Q.qnorm(Aop) @ Q.qnorm(Xh)
    err = Q.qnorm(host(Y)[:, rows.cpu().numpy(), :] - want)
    assert float((err / scale).max()) < 2.5e-5, float((err / scale).max())
