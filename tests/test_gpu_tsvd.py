"""Parity of the core truncated QSVD (Def. 1 eq. qsvd; "Truncated SVD(R, k)" of Algorithms
1, 2, 4) against the oracle's complex-adjoint QSVD."""
import numpy as np
import pytest

import synth
from oracle import quaternion as Q
from oracle.qr import qr
from oracle.qsvd import tsvd
from tests._qutil import np_to_small, small, small_to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    c = qlr.Context(0)
    yield c
    c.close()


def _upper_r(l, sig, seed):
    Uq, _ = qr(synth.gaussian_qmat(seed, l, l))
    Vq, _ = qr(synth.gaussian_qmat(seed + 1, l, l))
    X = Q.qmatmul(Uq * sig, Q.qH(Vq))
    _, R = qr(X)
    return R


def _proj(M):
    return Q.qmatmul(M, Q.qH(M))


@pytest.mark.parametrize("l,k,prec,decay", [(15, 10, 0, "geom"), (30, 30, 0, "geom"), (110, 100, 1, "harm"),
                                            (110, 100, 0, "harm"), (2, 1, 0, "geom"), (1, 1, 1, "geom"),
                                            (64, 20, 1, "exp"), (180, 50, 1, "harm")])
def test_core_tsvd_parity(ctx, l, k, prec, decay):
    from paper_2507_13731_gb300 import qlr
    i = np.arange(1, l + 1)
    sig = {"geom": 0.5 ** (i - 1), "harm": 1.0 / i, "exp": np.exp(-i / 20.0)}[decay]
    R = _upper_r(l, sig, 3 + l)
    Lw, Sw, Rw = tsvd(R, k)
    Rd = np_to_small(R)
    Ld, Sd, Rtd = small(l, k), small(1, k)[0, :, 0].contiguous(), small(l, k)
    import torch
    Sd = torch.zeros(k, dtype=torch.float64, device="cuda")
    qlr.qtsvd(ctx, Rd, k, Ld, Sd, Rtd, prec)
    assert ctx.sync() == 0
    S = Sd.cpu().numpy()
    L, Rt = small_to_np(Ld), small_to_np(Rtd)
    tol = 1e-11 if prec == 0 else 2e-6
    np.testing.assert_allclose(S, Sw, rtol=tol * (1 if prec == 0 else sig[0] / sig[k - 1]))
    # R v = sigma u and orthonormal vectors
    np.testing.assert_allclose(Q.qmatmul(R, Rt), L * S, atol=(1e-11 if prec == 0 else 1e-5) * sig[0])
    np.testing.assert_allclose(Q.qmatmul(Q.qH(Rt), Rt), Q.qeye(k), atol=1e-10 if prec == 0 else 1e-5)
    # subspace of the leading singular vectors up to a well separated gap
    gaps = sig[:k - 1] / sig[1:k]
    cut = next((j + 1 for j in range(k - 2, -1, -1) if gaps[j] > 1.2), None)
    if cut is not None:
        np.testing.assert_allclose(_proj(Rt[:, :, :cut]), _proj(Rw[:, :, :cut]),
                                   atol=1e-9 if prec == 0 else 1e-4)


def test_core_tsvd_repeated_values(ctx):
    import torch
    from paper_2507_13731_gb300 import qlr
    sig = np.array([2.0, 1.0, 1.0, 1.0, 0.5, 0.25])
    R = _upper_r(6, sig, 99)
    Ld, Rtd = small(6, 6), small(6, 6)
    Sd = torch.zeros(6, dtype=torch.float64, device="cuda")
    qlr.qtsvd(ctx, np_to_small(R), 6, Ld, Sd, Rtd, 0)
    assert ctx.sync() == 0
    np.testing.assert_allclose(Sd.cpu().numpy(), sig, rtol=1e-12)
    L, Rt = small_to_np(Ld), small_to_np(Rtd)
    np.testing.assert_allclose(Q.qmatmul(L * Sd.cpu().numpy(), Q.qH(Rt)), R, atol=1e-12)


def test_fp32_sweeps_match_fp64_core(ctx):
    """The core QSVD of the FP32 modes (FP32 one-sided Jacobi sweeps, then the kept triplets
    re-evaluated in FP64 as Rayleigh quotients of the FP64 R) against the FP64 core on the same R:
    l = 110, sigma_i = 1/i, k = 100 (the 4096 x 4096 workload's core).  Bounds: the singular values
    to 1e-6 relative (the refinement's error is second order in the vectors' angles, ~u32 / relgap
    with relative gaps >= 0.005 here); the rank-k projectors of both vector sets to 5e-4 entrywise
    (sin of the subspace angle <= eps / relgap_k with eps ~ 4 sqrt(l) u32 and relgap_k =
    (sigma_100 - sigma_101) / sigma_100 ~ 0.0099)."""
    import torch
    from paper_2507_13731_gb300 import qlr
    l, k = 110, 100
    sig = 1.0 / np.arange(1, l + 1)
    R = _upper_r(l, sig, 113)
    out = {}
    for prec in (qlr.F64, qlr.F32):
        Ld, Rtd = small(l, k), small(l, k)
        Sd = torch.zeros(k, dtype=torch.float64, device="cuda")
        qlr.qtsvd(ctx, np_to_small(R), k, Ld, Sd, Rtd, prec)
        assert ctx.sync() == 0
        out[prec] = (small_to_np(Ld), Sd.cpu().numpy(), small_to_np(Rtd))
    (L64, S64, R64), (L32, S32, R32) = out[qlr.F64], out[qlr.F32]
    np.testing.assert_allclose(S32, S64, rtol=1e-6)
    assert float(np.abs(_proj(R32) - _proj(R64)).max()) <= 5e-4
    assert float(np.abs(_proj(L32) - _proj(L64)).max()) <= 5e-4
