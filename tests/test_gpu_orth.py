"""Parity of the orthonormalisation step ("QR" of Def. 1, eq. QQR): FP64 Gram, quaternion
Cholesky, CholeskyQR2 and shifted CholeskyQR3, against the oracle's Householder QR (the thin QR
with real positive diag(R) is unique, so Q and R are compared element by element)."""
import numpy as np
import pytest
import torch

import synth
from oracle import quaternion as Q
from oracle.qr import qr
from tests._qutil import dev_thin, host, small, small_to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    c = qlr.Context(0)
    yield c
    c.close()


def _conditioned(m, l, cond, seed):
    Uq, _ = qr(synth.gaussian_qmat(seed, m, l))
    Vq, _ = qr(synth.gaussian_qmat(seed + 1, l, l))
    s = np.geomspace(1.0, 1.0 / cond, l)
    return Q.qmatmul(Uq * s, Q.qH(Vq))


@pytest.mark.parametrize("m,l,dt", [(1000, 37, "f32"), (333, 1, "f64"), (4096, 110, "f32"), (70, 70, "f64")])
def test_gram(ctx, m, l, dt):
    from paper_2507_13731_gb300 import qlr
    Y = synth.gaussian_qmat(5, m, l)
    Yd = dev_thin(Y, dt)
    G = small(l)
    qlr.qgram(ctx, Yd, G)
    assert ctx.sync() == 0
    Yh = host(Yd)
    want = Q.qmatmul(Q.qH(Yh), Yh)
    scale = Q.qnorm(Q.qH(Yh)) @ Q.qnorm(Yh)
    assert np.all(Q.qnorm(small_to_np(G) - want) <= 64 * m * 2.0 ** -53 * scale)


@pytest.mark.parametrize("m,l,seed", [(1, 1, 1), (513, 64, 2), (64, 200, 3), (2048, 17, 4), (4100, 110, 5)])
def test_gram_fp32_graded_normwise(ctx, m, l, seed):
    """FP32 Gram (tensor-core exact slicing when it applies) on columns scaled over 12 decades and
    rows over 6: every entry within 2^-36 sqrt(m) |y_i| |y_j| of the FP64 Gram of the stored data --
    FP64-class normwise, far below the 2^-24 of an FP32 sum.  Covers one row, chunk boundaries
    (513 rows), several W tiles (l = 200) and ragged tiles."""
    from paper_2507_13731_gb300 import qlr
    rng = np.random.default_rng(seed)
    Y = synth.gaussian_qmat(seed, m, l)
    Y = Y * (10.0 ** rng.uniform(-6, 6, size=l))[None, None, :] * (10.0 ** rng.uniform(-3, 3, size=m))[None, :, None]
    Yd = dev_thin(Y, "f32")
    G = small(l)
    qlr.qgram(ctx, Yd, G)
    assert ctx.sync() == 0
    Yh = host(Yd)
    want = Q.qmatmul(Q.qH(Yh), Yh)
    cn = np.sqrt((Yh ** 2).sum(axis=(0, 1)))
    Gh = small_to_np(G)
    assert np.all(Q.qnorm(Gh - want) <= 2.0 ** -36 * np.sqrt(m) * np.outer(cn, cn))
    assert np.all(Gh[1:, np.arange(l), np.arange(l)] == 0.0)


@pytest.mark.parametrize("l", [1, 5, 64, 110])
def test_chol_matches_unique_qr_factor(ctx, l):
    from paper_2507_13731_gb300 import qlr
    Y = _conditioned(3 * l + 10, l, 1e3, 7)
    _, Rw = qr(Y)
    G = Q.qmatmul(Q.qH(Y), Y)
    Gd = torch.from_numpy(np.ascontiguousarray(G.transpose(0, 2, 1))).cuda()
    Rd = small(l)
    qlr.qchol(ctx, Gd, Rd)
    assert ctx.sync() == 0
    np.testing.assert_allclose(small_to_np(Rd), Rw, atol=1e-9 * np.abs(Rw).max())


@pytest.mark.parametrize("m,l,cond,dt,orth", [(500, 23, 1e2, "f64", 0), (2000, 110, 1e3, "f32", 0),
                                             (300, 40, 1e10, "f64", 1), (1500, 60, 1e6, "f32", 1),
                                             (64, 64, 10.0, "f64", 0), (17, 3, 5.0, "f32", 0),
                                             (2000, 40, 3e4, "f32", 0), (3000, 110, 3e2, "f32", 0)])
def test_cholqr_parity(ctx, m, l, cond, dt, orth):
    """CholeskyQR2's second step uses the series factorisation when Q'^H Q' is close to I and the
    blocked Cholesky otherwise (the 3e4-conditioned FP32 case); both must give the unique QR."""
    from paper_2507_13731_gb300 import qlr
    Y = _conditioned(m, l, cond, 11)
    Yd = dev_thin(Y, dt)
    Yh = host(Yd)
    Qd = qlr.empty_thin(m, l, Yd.dtype)
    Rd = small(l)
    qlr.cholqr(ctx, Yd, Qd, Rd, orth)
    assert ctx.sync() == 0
    Qh, Rh = host(Qd), small_to_np(Rd)
    Qw, Rw = qr(Yh)
    u = 2.0 ** -53 if dt == "f64" else 2.0 ** -24
    orth_err = np.abs(Q.qmatmul(Q.qH(Qh), Qh) - Q.qeye(l)).max()
    assert orth_err <= 200 * l * u
    recon = Q.qfro(Q.qmatmul(Qh, Rh) - Yh) / Q.qfro(Yh)
    assert recon <= 50 * l * u * (cond if orth == 1 else 1.0)
    if cond * u < 1e-3:   # well conditioned: unique factors agree element by element
        tol = 50 * l * u * cond
        np.testing.assert_allclose(Rh, Rw, atol=tol * np.abs(Rw).max())
        np.testing.assert_allclose(Qh, Qw, atol=tol)


def test_cholqr2_breakdown_is_reported(ctx):
    from paper_2507_13731_gb300 import qlr
    Y = synth.gaussian_qmat(3, 50, 6)
    Y[:, :, 4] = 0.0
    Yd = dev_thin(Y, "f64")
    Qd = qlr.empty_thin(50, 6, torch.float64)
    qlr.cholqr(ctx, Yd, Qd, None, qlr.ORTH_CHOLQR2)
    assert ctx.sync() == qlr.ENOTPD
    assert ctx.sync() == 0          # the error word is cleared once read
