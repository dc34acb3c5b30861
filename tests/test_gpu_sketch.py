"""Parity of the sketch products Y = A X and Z = A^H Y (eq. 1 summed over the inner index;
X^H of Section 2) against the FP64 oracle, element by element."""
import numpy as np
import pytest

import synth
from oracle import quaternion as Q
from tests._qutil import dev_rowmajor, dev_thin, host

pytestmark = pytest.mark.gpu

U32, U64 = 2.0 ** -24, 2.0 ** -53


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    c = qlr.Context(0)
    yield c
    c.close()


def _abs_bound(A, X):
    """sum_k |a_ik| |x_kj| with quaternion norms (entrywise error scale of the product)."""
    return Q.qnorm(A) @ Q.qnorm(X)


SHAPES = [(200, 150, 13, False), (64, 64, 16, False), (1, 1, 1, False), (300, 257, 37, True),
          (129, 1000, 5, False), (1000, 129, 112, False), (17, 33, 128, True)]


@pytest.mark.parametrize("m,n,l,pure", SHAPES)
@pytest.mark.parametrize("compute,dt,u", [("F64", "f64", U64), ("F32", "f32", U32)])
@pytest.mark.parametrize("op", ["N", "H"])
def test_sketch_simt_parity(ctx, m, n, l, pure, compute, dt, u, op):
    from paper_2507_13731_gb300 import qlr
    A = synth.gaussian_qmat(11 + m, m, n)
    if pure:
        A[0] = 0.0
    rows_in = n if op == "N" else m
    X = synth.gaussian_qmat(12 + n, rows_in, l)
    Ad = dev_rowmajor(A, dt, pure=pure)
    Xd = dev_thin(X, dt)
    Ah, Xh = host(Ad), host(Xd)                       # the values the GPU actually sees
    rows_out = m if op == "N" else n
    Yd = qlr.empty_thin(rows_out, l, Xd.dtype)
    qlr.qsketch(ctx, qlr.OP_N if op == "N" else qlr.OP_H, Ad, Xd, Yd, getattr(qlr, "COMPUTE_" + compute))
    assert ctx.sync() == 0
    Aop = Ah if op == "N" else Q.qH(Ah)
    want = Q.qmatmul(Aop, Xh)
    bound = 8 * rows_in * u * _abs_bound(Aop, Xh) + 1e-300
    err = Q.qnorm(host(Yd) - want)
    assert np.all(err <= bound), float((err / bound).max())


def test_sketch_full_size_sampled_rows(ctx):
    """Slow-decay 4096 x 4096 FP32 workload, l = 110: sampled output rows against the oracle."""
    from paper_2507_13731_gb300 import qlr
    P = synth.config_slow_decay(4096, 4096, 100, 10, 4)
    Ad, Xd = dev_rowmajor(P.A, "f32"), dev_thin(P.Omega, "f32")
    rng = np.random.default_rng(0)
    rows = rng.choice(4096, 64, replace=False)
    for op in (qlr.OP_N, qlr.OP_H):
        Yd = qlr.empty_thin(4096, 110)
        qlr.qsketch(ctx, op, Ad, Xd, Yd, qlr.COMPUTE_F32)
        assert ctx.sync() == 0
        Ah = host(Ad)
        Aop = Ah[:, rows, :] if op == qlr.OP_N else Q.qH(Ah)[:, rows, :]
        want = Q.qmatmul(Aop, host(Xd))
        bound = 8 * 4096 * U32 * _abs_bound(Aop, host(Xd))
        assert np.all(Q.qnorm(host(Yd)[:, rows, :] - want) <= bound)


def test_sketch_rejects_bad_arguments(ctx):
    import torch
    from paper_2507_13731_gb300 import qlr
    A = torch.zeros(4, 8, 6, device="cuda")
    X = qlr.empty_thin(5, 3)
    Y = qlr.empty_thin(8, 3)
    with pytest.raises(qlr.QlrError) as e:
        qlr.qsketch(ctx, qlr.OP_N, A, X, Y, qlr.COMPUTE_F32)
    assert e.value.code == qlr.ESHAPE
    X = qlr.empty_thin(6, 3, torch.float64)
    with pytest.raises(qlr.QlrError) as e:
        qlr.qsketch(ctx, qlr.OP_N, A, X, Y, qlr.COMPUTE_F32)
    assert e.value.code == qlr.EINVAL
