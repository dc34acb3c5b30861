"""Full-size parity at the five workload configurations, in the launch configuration bench.py
uses (AUTO compute, context workspace), against the FP64 oracle run on the same Omega and the
unrounded A.  Tolerances on singular values (relative): 1e-10 in FP64, 1e-4 in FP32 (3xTF32),
2e-2 in BF16 and in single-product TF32 (10-bit mantissa, between BF16 and FP32)."""
import numpy as np
import pytest
import torch

import synth
from oracle import algorithms as al
from oracle import quaternion as Q
from tests._qutil import dev_rowmajor, dev_thin, host

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    c = qlr.Context(0)
    yield c
    c.close()


def _run(ctx, P, v, dt, compute, algo=None, A_dev=None):
    from paper_2507_13731_gb300 import qlr
    Ad = A_dev if A_dev is not None else dev_rowmajor(P.A, dt, pure=P.pure)
    Od = dev_thin(P.Omega, "f64" if dt == "f64" else "f32")
    tdt = torch.float64 if dt == "f64" else torch.float32
    U, V = qlr.empty_thin(P.m, P.k, tdt), qlr.empty_thin(P.n, P.k, tdt)
    S = torch.zeros(P.k, dtype=torch.float64, device="cuda")
    qlr.qsvd_lowrank(ctx, Ad, P.k, P.p, v, Od, U, S, V, algo=algo or qlr.ALG2, compute=compute, side=qlr.SIDE_X)
    assert ctx.sync() == 0
    return host(U), S.cpu().numpy(), host(V), Ad


def _orth_err(M):
    return float(np.abs(Q.qmatmul(Q.qH(M), M) - Q.qeye(M.shape[2])).max())


@pytest.fixture(scope="module")
def config2():
    return synth.config2(4)


@pytest.mark.parametrize("v", [2, 3, 4, 6, 8])
def test_config2_fp32_all_pass_budgets(ctx, config2, v):
    """4096 x 4096, FP32 planes, sigma_i = 1/i, k = 100, p = 10: the bench workload."""
    from paper_2507_13731_gb300 import qlr
    P = config2
    U, S, V, _ = _run(ctx, P, v, "f32", qlr.COMPUTE_AUTO)
    ref = al.alg2_arbitrary_pass(P.A, P.k, P.p, v, P.Omega)
    np.testing.assert_allclose(S, ref.S, rtol=1e-4)
    assert _orth_err(U) < 1e-5 and _orth_err(V) < 1e-5


def test_config3_bf16_full_size():
    """16384 x 8192 quaternion in BF16 planes (~1 GB), sigma_i = exp(-i/50), k = 200, p = 20, v = 4,
    BF16 sketches with FP32 accumulation, FP64-class Gram / Cholesky / core QSVD."""
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    c = qlr.Context(0)
    P = synth.config3()
    U, S, V, _ = _run(c, P, 4, "bf16", qlr.COMPUTE_AUTO)
    ref = al.alg2_arbitrary_pass(P.A, P.k, P.p, 4, P.Omega)
    np.testing.assert_allclose(S, ref.S, rtol=2e-2)
    assert _orth_err(U) < 1e-4 and _orth_err(V) < 1e-4
    c.close()


@pytest.mark.parametrize("compute,tol", [("TF32X3", 1e-4), ("TF32_MIXED", 1e-4), ("TF32", 2e-2)])
def test_config4_block_krylov_full_size(ctx, compute, tol):
    """20000 x 10000 pure quaternion colour field, Algorithm 4 with k = 50, b = 60, v = 6: the top-k
    singular values within the FP32 tolerance 1e-4 of the FP64 oracle's on the unrounded A in
    3xTF32 and in the mixed mode (one TF32 product for the Krylov blocks, 3xTF32 for the final
    pass), 2e-2 with single-product TF32 throughout.  The field's leading singular value is ~9x
    the next, so the plain stack of Krylov blocks is numerically rank-deficient in FP32 (the oracle
    pin test_alg4_fp32_rounding_floor_on_colour_field); the GPU deflates each new block against the
    earlier ones, which keeps the directions the stack adds (same span in exact arithmetic)."""
    from paper_2507_13731_gb300 import qlr
    P = _config4()
    U, S, V, _ = _run(ctx, P, 6, "f32", getattr(qlr, "COMPUTE_" + compute), algo=qlr.ALG4,
                      A_dev=_config4_dev())
    ref = _config4_ref()
    np.testing.assert_allclose(S, ref.S, rtol=tol)
    assert _orth_err(U) < 1e-4 and _orth_err(V) < 1e-4


_C4 = {}


def _config4():
    if "P" not in _C4:
        _C4["P"] = synth.config4()
    return _C4["P"]


def _config4_dev():
    if "A" not in _C4:
        _C4["A"] = dev_rowmajor(_config4().A, "f32", pure=True)
    return _C4["A"]


def _config4_ref():
    if "ref" not in _C4:
        P = _config4()
        _C4["ref"] = al.alg4_block_flexible(P.A, P.k, P.p, 6, P.Omega)
    return _C4["ref"]


def test_config5_batched_bf16_sampled(ctx):
    """512 pure matrices of uneven sizes (64..1024 x 64..768), rank 8..64 plus noise, k = r,
    p = 8, v = 3, BF16 storage with a 16-byte row pitch: one batch plan (grouped tensor-core
    sketch per pass, CUDA graph), every matrix on the GPU, 24 sampled ones against the oracle;
    a replay of the graph reproduces the first run."""
    from paper_2507_13731_gb300 import qlr
    probs = synth.batched_problems()
    As = []
    for P in probs:
        t = qlr.empty_rowmajor(P.m, P.n, 3, torch.bfloat16)
        t.copy_(torch.from_numpy(np.ascontiguousarray(P.A[1:])).to(torch.bfloat16))
        As.append(t)
    Os = [dev_thin(P.Omega, "f32") for P in probs]
    Us = [qlr.empty_thin(P.m, P.k) for P in probs]
    Vs = [qlr.empty_thin(P.n, P.k) for P in probs]
    Ss = [torch.zeros(P.k, dtype=torch.float64, device="cuda") for P in probs]
    b = qlr.Batch(ctx, As, [P.k for P in probs], [P.p for P in probs], 3, Os, Us, Ss, Vs)
    assert ctx.sync() == 0
    first = [s.clone() for s in Ss]
    b.run()
    assert ctx.sync() == 0
    for s, f in zip(Ss, first):
        np.testing.assert_allclose(s.cpu().numpy(), f.cpu().numpy(), rtol=1e-12, atol=0)
    rng = np.random.default_rng(5)
    for i in rng.choice(len(probs), 24, replace=False):
        P = probs[i]
        ref = al.alg2_arbitrary_pass(P.A, P.k, P.p, 3, P.Omega)
        np.testing.assert_allclose(Ss[i].cpu().numpy(), ref.S, rtol=2e-2, err_msg=f"problem {i}")
    b.close()
