"""End-to-end parity of Algorithm 2 / Algorithm 4 against the oracle run on the same Omega."""
import numpy as np
import pytest
import torch

import synth
from oracle import algorithms as al
from oracle import norms
from oracle import quaternion as Q
from oracle.qsvd import singular_values
from tests._qutil import dev_rowmajor, dev_thin, host, small, small_to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    c = qlr.Context(0)
    yield c
    c.close()


def _proj(M):
    return Q.qmatmul(M, Q.qH(M))


def run_gpu(ctx, P, v, algo, dt, compute, side=None, Ad=None):
    from paper_2507_13731_gb300 import qlr
    side = qlr.SIDE_X if side is None else side
    if Ad is None:
        Ad = dev_rowmajor(P.A, dt, pure=P.pure)
    Om = P.Omega if side == qlr.SIDE_X else synth.omega_for(77, P.m, P.ell)
    Od = dev_thin(Om, "f64" if dt == "f64" else "f32")
    tdt = torch.float64 if dt == "f64" else torch.float32
    U, V = qlr.empty_thin(P.m, P.k, tdt), qlr.empty_thin(P.n, P.k, tdt)
    S = torch.zeros(P.k, dtype=torch.float64, device="cuda")
    qlr.qsvd_lowrank(ctx, Ad, P.k, P.p, v, Od, U, S, V, algo=algo, compute=compute, side=side)
    assert ctx.sync() == 0
    return host(U), S.cpu().numpy(), host(V), Om, Ad


@pytest.mark.parametrize("v", [2, 3, 4, 5])
def test_config1_fp64_alg2(ctx, v):
    from paper_2507_13731_gb300 import qlr
    P = synth.config1()
    U, S, V, Om, _ = run_gpu(ctx, P, v, qlr.ALG2, "f64", qlr.COMPUTE_F64)
    ref = al.alg2_arbitrary_pass(P.A, P.k, P.p, v, Om)
    np.testing.assert_allclose(S, ref.S, rtol=1e-10)
    np.testing.assert_allclose(_proj(U[:, :, :8]), _proj(ref.U[:, :, :8]), atol=1e-8)
    np.testing.assert_allclose(_proj(V[:, :, :8]), _proj(ref.V[:, :, :8]), atol=1e-8)


@pytest.mark.parametrize("algo", ["alg2", "alg4"])
@pytest.mark.parametrize("v", [4, 7])
def test_qr_every_pass_flag(ctx, algo, v):
    """Both settings of QLR_FLAG_QR_EVERY_PASS give the oracle's singular values to 1e-10 and the
    same rank-k subspaces: the intermediate bases differ only by l x l rotations."""
    from paper_2507_13731_gb300 import qlr
    P = synth.config_slow_decay(300, 220, 12, 6, v, seed=26)
    Ad = dev_rowmajor(P.A, "f64")
    Od = dev_thin(P.Omega, "f64")
    a = qlr.ALG2 if algo == "alg2" else qlr.ALG4
    ref = (al.alg2_arbitrary_pass if algo == "alg2" else al.alg4_block_flexible)(P.A, 12, 6, v, P.Omega)
    for every in (True, False):
        U, V = qlr.empty_thin(300, 12, torch.float64), qlr.empty_thin(220, 12, torch.float64)
        S = torch.zeros(12, dtype=torch.float64, device="cuda")
        qlr.qsvd_lowrank(ctx, Ad, 12, 6, v, Od, U, S, V, algo=a, compute=qlr.COMPUTE_F64, side=qlr.SIDE_X,
                         qr_every_pass=every)
        assert ctx.sync() == 0
        np.testing.assert_allclose(S.cpu().numpy(), ref.S, rtol=1e-10)
        np.testing.assert_allclose(_proj(host(U)[:, :, :8]), _proj(ref.U[:, :, :8]), atol=1e-8)


@pytest.mark.parametrize("algo,q", [("alg1", 0), ("alg1", 1), ("alg1", 2), ("alg3", 1), ("alg3", 2)])
def test_classical_algorithms_match_oracle(ctx, algo, q):
    """QLR_ALG1 / QLR_ALG3 with 2q + 2 passes against the oracle's Algorithm 1 (power scheme, a QR
    after every product) and Algorithm 3 (one QR of the stacked Krylov matrix, full SVD of Q^H X)
    on the same Omega: singular values to 1e-9, rank-8 subspaces to 1e-8.  An odd pass count is
    rejected with QLR_ESHAPE."""
    from paper_2507_13731_gb300 import qlr
    v = 2 * q + 2
    P = synth.config_slow_decay(300, 220, 12, 6, v, seed=31 + q)
    a = qlr.ALG1 if algo == "alg1" else qlr.ALG3
    U, S, V, Om, Ad = run_gpu(ctx, P, v, a, "f64", qlr.COMPUTE_F64)
    ref = (al.alg1_classical if algo == "alg1" else al.alg3_block_classical)(P.A, P.k, P.p, q, Om)
    np.testing.assert_allclose(S, ref.S, rtol=1e-9)
    np.testing.assert_allclose(_proj(U[:, :, :8]), _proj(ref.U[:, :, :8]), atol=1e-8)
    np.testing.assert_allclose(_proj(V[:, :, :8]), _proj(ref.V[:, :, :8]), atol=1e-8)
    Od = dev_thin(Om, "f64")
    Ub, Vb = qlr.empty_thin(P.m, P.k, torch.float64), qlr.empty_thin(P.n, P.k, torch.float64)
    Sb = torch.zeros(P.k, dtype=torch.float64, device="cuda")
    with pytest.raises(qlr.QlrError):
        qlr.qsvd_lowrank(ctx, Ad, P.k, P.p, v + 1, Od, Ub, Sb, Vb, algo=a, compute=qlr.COMPUTE_F64, side=qlr.SIDE_X)


@pytest.mark.parametrize("algo,v", [("alg2", 2), ("alg2", 3), ("alg1", 4), ("alg1", 6)])
def test_random_lowrank_example(ctx, algo, v):
    """The random low-rank example (Section 8): A = B C of exact rank 50, m = n = 500, FP32 planes
    with 3xTF32 sketches; Algorithm 2 with two and three passes and Algorithm 1 with q = 1, 2
    against the oracle on the same Omega (sigma to 1e-4), and the rank-50 approximation
    reproduces A to FP32 rounding (Frobenius relative error below 1e-5)."""
    from paper_2507_13731_gb300 import qlr
    P = synth.random_lowrank_problem(500, 500, 50, v=v)
    a = qlr.ALG1 if algo == "alg1" else qlr.ALG2
    U, S, V, Om, _ = run_gpu(ctx, P, v, a, "f32", qlr.COMPUTE_TF32X3)
    ref = (al.alg1_classical(P.A, P.k, P.p, v // 2 - 1, Om) if algo == "alg1"
           else al.alg2_arbitrary_pass(P.A, P.k, P.p, v, Om))
    np.testing.assert_allclose(S, ref.S, rtol=1e-4)
    X = Q.qmatmul(U * S[None, None, :], Q.qH(V))
    assert Q.qfro(X - P.A) <= 1e-5 * Q.qfro(P.A)


@pytest.mark.parametrize("v", [2, 3, 4, 5, 6])
def test_alg4_fp64_small(ctx, v):
    from paper_2507_13731_gb300 import qlr
    P = synth.config_slow_decay(160, 120, 6, 4, v, seed=21)
    U, S, V, Om, _ = run_gpu(ctx, P, v, qlr.ALG4, "f64", qlr.COMPUTE_F64)
    ref = al.alg4_block_flexible(P.A, 6, 4, v, Om)
    np.testing.assert_allclose(S, ref.S, rtol=1e-9)
    err_gpu = norms.lowrank_error(P.A, U, S, V)
    err_ref = norms.lowrank_error(P.A, ref.U, ref.S, ref.V)
    assert abs(err_gpu - err_ref) <= 1e-8 * err_ref


@pytest.mark.parametrize("compute,tol", [("F32", 1e-4), ("TF32_MIXED", 1e-4), ("TF32_RN", 1e-3)])
@pytest.mark.parametrize("v", [2, 3, 4])
def test_fp32_slow_decay(ctx, v, compute, tol):
    """Algorithm 2 with FP32 storage: plain FP32 (SIMT) and the mixed mode (TF32 products for the
    passes that only feed the next basis, 3xTF32 for the last pass) within the FP32 tolerance 1e-4
    of the oracle's singular values; the rounded-TF32 mode (the last pass one product of operands
    rounded to nearest TF32: op N for odd v, op H for even v) within 1e-3.  This matrix's singular
    vectors are concentrated on few entries (a unit-quaternion diagonal and 8 reflectors per side),
    so the rounding of those entries (2^-12 relative) moves sigma_1 at first order: a CPU model of
    the same arithmetic gives 2e-4..4e-4, where 3xTF32 gives 4e-5."""
    from paper_2507_13731_gb300 import qlr
    P = synth.config_slow_decay(1024, 768, 40, 10, v, seed=22)
    U, S, V, Om, _ = run_gpu(ctx, P, v, qlr.ALG2, "f32", getattr(qlr, "COMPUTE_" + compute))
    ref = al.alg2_arbitrary_pass(P.A, 40, 10, v, Om)
    np.testing.assert_allclose(S, ref.S, rtol=tol)


@pytest.mark.parametrize("v", [2, 3])
def test_side_xh(ctx, v):
    from paper_2507_13731_gb300 import qlr
    P = synth.config_slow_decay(90, 140, 8, 4, v, seed=23)
    U, S, V, Om, _ = run_gpu(ctx, P, v, qlr.ALG2, "f64", qlr.COMPUTE_F64, side=qlr.SIDE_XH)
    ref = al.run("alg2", P.A, 8, 4, v, Om, side="XH")
    np.testing.assert_allclose(S, ref.S, rtol=1e-10)
    np.testing.assert_allclose(_proj(U[:, :, :6]), _proj(ref.U[:, :, :6]), atol=1e-8)


@pytest.mark.parametrize("every_pass", [True, False])
def test_rangefinder_factors(ctx, every_pass):
    """With a QR at every pass the factors equal the oracle's; by default the bases that only feed
    the next pass get one shifted CholeskyQR step, so Q1, Q2, R equal the oracle's up to unitary
    l x l rotations: same projectors, same singular values of R, same defining relation."""
    from paper_2507_13731_gb300 import qlr
    P = synth.config_slow_decay(200, 150, 10, 5, 3, seed=24)
    Ad = dev_rowmajor(P.A, "f64")
    Od = dev_thin(P.Omega, "f64")
    Q1, Q2 = qlr.empty_thin(200, 15, torch.float64), qlr.empty_thin(150, 15, torch.float64)
    R = small(15)
    for v in (2, 3, 4, 5):
        side = qlr.qrangefinder(ctx, Ad, 10, 5, v, Od, Q1, Q2, R, compute=qlr.COMPUTE_F64, side=qlr.SIDE_X,
                                qr_every_pass=every_pass)
        assert ctx.sync() == 0 and side == qlr.SIDE_X
        ref = al.alg2_arbitrary_pass(P.A, 10, 5, v, P.Omega)
        q1, q2, r = host(Q1), host(Q2), small_to_np(R)
        if every_pass or v == 2:
            np.testing.assert_allclose(q1, ref.Q1, atol=1e-9)
            np.testing.assert_allclose(r, ref.R, atol=1e-10)
            np.testing.assert_allclose(q2, ref.Q2, atol=1e-9)
            continue
        for q, rq in ((q1, ref.Q1), (q2, ref.Q2)):
            np.testing.assert_allclose(Q.qmatmul(q, Q.qH(q)), Q.qmatmul(rq, Q.qH(rq)), atol=1e-9)
        np.testing.assert_allclose(singular_values(r), singular_values(ref.R), rtol=1e-10, atol=1e-12)
        # odd v: X Q2 = Q1 R1; even v: X^H Q1 = Q2 R2
        lhs = Q.qmatmul(P.A, q2) if v % 2 else Q.qmatmul(Q.qH(P.A), q1)
        rhs = Q.qmatmul(q1, r) if v % 2 else Q.qmatmul(q2, r)
        np.testing.assert_allclose(lhs, rhs, atol=1e-9)


def test_batched_loop_pure(ctx):
    from paper_2507_13731_gb300 import qlr
    probs = synth.batched_problems(count=4, mmax=200, nmax=150, rmax=12)
    As = [dev_rowmajor(P.A, "f32", pure=True) for P in probs]
    Os = [dev_thin(P.Omega, "f32") for P in probs]
    Us = [qlr.empty_thin(P.m, P.k) for P in probs]
    Vs = [qlr.empty_thin(P.n, P.k) for P in probs]
    Ss = [torch.zeros(P.k, dtype=torch.float64, device="cuda") for P in probs]
    qlr.qsvd_lowrank_batched(ctx, As, [P.k for P in probs], [P.p for P in probs], 3, Os, Us, Ss, Vs,
                             compute=qlr.COMPUTE_F32)
    assert ctx.sync() == 0
    for P, S in zip(probs, Ss):
        ref = al.alg2_arbitrary_pass(P.A, P.k, P.p, 3, P.Omega)
        np.testing.assert_allclose(S.cpu().numpy(), ref.S, rtol=1e-4)


def test_residual_norm_matches_oracle(ctx):
    from paper_2507_13731_gb300 import qlr
    P = synth.config_slow_decay(300, 200, 10, 5, 2, seed=25)
    ref = al.alg2_arbitrary_pass(P.A, 10, 5, 2, P.Omega)
    Ad = dev_rowmajor(P.A, "f64")
    start = dev_thin(synth.gaussian_qmat(9, 200, 6), "f64")
    e1 = qlr.residual_norm(ctx, Ad, dev_thin(ref.Q1, "f64"), qlr.SIDE_X, start, iters=60)
    e2 = qlr.residual_norm(ctx, Ad, dev_thin(ref.Q2, "f64"), qlr.SIDE_XH, start, iters=60)
    w1, w2 = norms.range_error(P.A, ref.Q1), norms.corange_error(P.A, ref.Q2)
    assert w1 * (1 - 1e-3) <= e1 <= w1 * (1 + 1e-10)
    assert w2 * (1 - 1e-3) <= e2 <= w2 * (1 + 1e-10)


@pytest.mark.parametrize("v", [2, 3, 4, 5, 6, 7])
def test_alg4_basis_spans_oracle_krylov_space(ctx, v):
    """qlr_qbasis with Algorithm 4 (FP64): the stacked basis (Q1 = QR(K1) for even v, Q2 = QR(K2)
    for odd v, each new Krylov block deflated against the earlier ones on the GPU) spans the
    oracle's stacked Krylov space, so the projectors, the singular values of R and the defining
    relation (X^H Q1 = Q2 R2 / X Q2 = Q1 R1) agree with the oracle's Algorithm 4."""
    from paper_2507_13731_gb300 import qlr
    P = synth.config_slow_decay(240, 180, 8, 4, v, seed=40 + v)
    l = P.k + P.p
    L = qlr.stacked_width(qlr.ALG4, l, v)
    Ad = dev_rowmajor(P.A, "f64")
    Od = dev_thin(P.Omega, "f64")
    Q1, Q2 = qlr.empty_thin(P.m, L, torch.float64), qlr.empty_thin(P.n, L, torch.float64)
    R = small(L)
    side = qlr.qbasis(ctx, Ad, P.k, P.p, v, Od, Q1, Q2, R, algo=qlr.ALG4, compute=qlr.COMPUTE_F64,
                      side=qlr.SIDE_X)
    assert ctx.sync() == 0 and side == qlr.SIDE_X
    ref = al.alg4_block_flexible(P.A, P.k, P.p, v, P.Omega)
    q1, q2, r = host(Q1), host(Q2), small_to_np(R)
    for q, rq in ((q1, ref.Q1), (q2, ref.Q2)):
        np.testing.assert_allclose(Q.qmatmul(Q.qH(q), q), Q.qeye(L), atol=1e-12)
        np.testing.assert_allclose(_proj(q), _proj(rq), atol=1e-9)
    np.testing.assert_allclose(singular_values(r), singular_values(ref.R), rtol=1e-9, atol=1e-12)
    lhs = Q.qmatmul(P.A, q2) if v % 2 else Q.qmatmul(Q.qH(P.A), q1)
    rhs = Q.qmatmul(q1, r) if v % 2 else Q.qmatmul(q2, r)
    np.testing.assert_allclose(lhs, rhs, atol=1e-9 * np.abs(P.A).max() * P.m)


@pytest.mark.parametrize("compute", ["TF32X3", "F32", "TF32_MIXED", "TF32_RN"])
def test_alg4_fp32_colour_field(ctx, compute):
    """Algorithm 4 with FP32 storage on a colour field (the config-4 construction at 1200 x 600,
    k = 30, b = 40, v = 6): the top-k singular values within the FP32 tolerance 1e-4 of the FP64
    oracle's on the unrounded A.  The field's leading singular value is ~10x the next, so the
    plain stack of Krylov blocks is numerically rank-deficient at FP32 (the oracle pin
    test_alg4_fp32_rounding_floor_on_colour_field shows 2e-4..2e-3 from FP32 rounding alone); the
    GPU deflates each new block against the earlier ones, which keeps the new directions."""
    from paper_2507_13731_gb300 import qlr
    P = synth.config_colour(1200, 600, 30, 40, 6, seed=1237)
    U, S, V, Om, _ = run_gpu(ctx, P, 6, qlr.ALG4, "f32", getattr(qlr, "COMPUTE_" + compute))
    ref = al.alg4_block_flexible(P.A, P.k, P.p, 6, Om)
    np.testing.assert_allclose(S, ref.S, rtol=1e-4)


def test_seeded_omega_on_the_device(ctx):
    """qlr_fill_omega writes the seeded Gaussian test matrix (Def. 2) into a device matrix: the
    same Omega as the input module's, so a C caller that only has the seed runs the oracle's
    problem (config 1, FP64: singular values to 1e-10)."""
    from paper_2507_13731_gb300 import qlr
    P = synth.config1()
    Od = qlr.empty_thin(P.n, P.ell, torch.float64)
    qlr.fill_omega(ctx, qlr.splitmix64(1234, synth.TAG_OMEGA), Od)
    np.testing.assert_allclose(host(Od), P.Omega, rtol=1e-13, atol=1e-13)
    O32 = qlr.empty_thin(P.n, P.ell, torch.float32)
    qlr.fill_omega(ctx, qlr.splitmix64(1234, synth.TAG_OMEGA), O32)
    np.testing.assert_allclose(host(O32), P.Omega.astype(np.float32), rtol=1e-7, atol=1e-7)
    Ad = dev_rowmajor(P.A, "f64")
    U, V = qlr.empty_thin(P.m, P.k, torch.float64), qlr.empty_thin(P.n, P.k, torch.float64)
    S = torch.zeros(P.k, dtype=torch.float64, device="cuda")
    qlr.qsvd_lowrank(ctx, Ad, P.k, P.p, P.v, Od, U, S, V, compute=qlr.COMPUTE_F64, side=qlr.SIDE_X)
    assert ctx.sync() == 0
    ref = al.alg2_arbitrary_pass(P.A, P.k, P.p, P.v, P.Omega)
    np.testing.assert_allclose(S.cpu().numpy(), ref.S, rtol=1e-10)
