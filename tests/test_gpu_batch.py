"""Batch plans: grouped tensor-core sketch launches over many problems, per-problem
orthonormalisation lanes, CUDA graph replay and the tile-order autotuner, against the FP64
oracle run problem by problem on the same Omega (Algorithm 2)."""
import numpy as np
import pytest
import torch

import synth
from oracle import algorithms as al
from tests._qutil import dev_thin

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    c = qlr.Context(0)
    yield c
    c.close()


def _padded(P, dtype):
    from paper_2507_13731_gb300 import qlr
    planes = 3 if P.pure else 4
    t = qlr.empty_rowmajor(P.m, P.n, planes, dtype)
    src = P.A[1:] if P.pure else P.A
    t.copy_(torch.from_numpy(np.ascontiguousarray(src)).to(dtype))
    return t


def _buffers(probs, dtype):
    from paper_2507_13731_gb300 import qlr
    As = [_padded(P, dtype) for P in probs]
    Os = [dev_thin(P.Omega, "f32") for P in probs]
    Us = [qlr.empty_thin(P.m, P.k) for P in probs]
    Vs = [qlr.empty_thin(P.n, P.k) for P in probs]
    Ss = [torch.zeros(P.k, dtype=torch.float64, device="cuda") for P in probs]
    return As, Os, Us, Vs, Ss


def _orth_err(U):
    from oracle import quaternion as Q
    from tests._qutil import host
    h = host(U)
    return float(np.abs(Q.qmatmul(Q.qH(h), h) - Q.qeye(h.shape[2])).max())


@pytest.mark.parametrize("v", [2, 3, 4])
def test_batched_bf16_matches_oracle(ctx, v):
    """12 pure problems of uneven sizes (BF16 storage, padded row pitch) through the one-shot
    batched call, which plans the grouped path: sigma within 2e-2 of the FP64 oracle."""
    from paper_2507_13731_gb300 import qlr
    probs = synth.batched_problems(count=12, seed=41, mmax=400, nmax=300, rmax=24, v=v)
    As, Os, Us, Vs, Ss = _buffers(probs, torch.bfloat16)
    qlr.qsvd_lowrank_batched(ctx, As, [P.k for P in probs], [P.p for P in probs], v, Os, Us, Ss, Vs)
    assert ctx.sync() == 0
    for i, P in enumerate(probs):
        ref = al.alg2_arbitrary_pass(P.A, P.k, P.p, v, P.Omega)
        np.testing.assert_allclose(Ss[i].cpu().numpy(), ref.S, rtol=2e-2, err_msg=f"problem {i}")
        assert _orth_err(Us[i]) < 1e-4 and _orth_err(Vs[i]) < 1e-4


def test_batch_plan_graph_replay(ctx):
    """A plan captured into a CUDA graph: every replay reproduces the first run's result, the
    autotuner has timed every grouped sketch variant, and a pass is two grouped launches."""
    from paper_2507_13731_gb300 import qlr
    probs = synth.batched_problems(count=20, seed=42, mmax=520, nmax=380, rmax=40)
    As, Os, Us, Vs, Ss = _buffers(probs, torch.bfloat16)
    b = qlr.Batch(ctx, As, [P.k for P in probs], [P.p for P in probs], 3, Os, Us, Ss, Vs)
    assert ctx.sync() == 0
    first = [s.clone() for s in Ss]
    info = b.info()
    assert info["graph"] and info["sketch_launches"] == 6 and 0 <= info["tile_order"] < 16
    timed = [v for v in range(16) if info["tune_ms"][v] > 0]
    # every schedule x order, and for the persistent one every tile shape (BF16: 2 + 8 variants)
    assert len(timed) == 10 and info["tune_ms"][info["tile_order"]] == min(info["tune_ms"][v] for v in timed)
    assert info["stage_k"] in (32, 64) and info["col_block_max"] % 16 == 0 and info["ring_stages"] >= 2
    assert info["launches_per_run"] > 6
    for _ in range(2):
        for s in Ss:
            s.zero_()
        b.run()
        assert ctx.sync() == 0
        for s, f in zip(Ss, first):
            np.testing.assert_allclose(s.cpu().numpy(), f.cpu().numpy(), rtol=1e-12, atol=0)
    for i in (0, 7, 19):
        P = probs[i]
        ref = al.alg2_arbitrary_pass(P.A, P.k, P.p, 3, P.Omega)
        np.testing.assert_allclose(Ss[i].cpu().numpy(), ref.S, rtol=2e-2, err_msg=f"problem {i}")
    b.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 6, 7, 10, 11, 14, 15])
def test_batch_sketch_variants(ctx, monkeypatch, variant):
    """Every grouped sketch variant (tile order x one CTA per tile / persistent CTAs x, for the
    persistent CTAs, 64- or 128-byte stage rows and column blocks of at most 128 or 64; fixed
    through QLR_BATCH_VARIANT) gives the oracle's sigma; 80 problems give the persistent CTAs
    several tiles each and exercise the alternating accumulators."""
    from paper_2507_13731_gb300 import qlr
    monkeypatch.setenv("QLR_BATCH_VARIANT", str(variant))
    probs = synth.batched_problems(count=80, seed=45, mmax=900, nmax=600, rmax=40)
    As, Os, Us, Vs, Ss = _buffers(probs, torch.bfloat16)
    b = qlr.Batch(ctx, As, [P.k for P in probs], [P.p for P in probs], 3, Os, Us, Ss, Vs, graph=False)
    assert ctx.sync() == 0 and b.info()["tile_order"] == variant
    for i in (0, 13, 27, 79):
        P = probs[i]
        ref = al.alg2_arbitrary_pass(P.A, P.k, P.p, 3, P.Omega)
        np.testing.assert_allclose(Ss[i].cpu().numpy(), ref.S, rtol=2e-2, err_msg=f"problem {i}")
    b.close()


def test_batch_plan_tf32x3_fp32(ctx):
    """FP32 storage with the 3xTF32 grouped sketch, eager runs (no graph): sigma within 1e-4."""
    from paper_2507_13731_gb300 import qlr
    probs = synth.batched_problems(count=9, seed=43, mmax=300, nmax=260, rmax=16)
    As, Os, Us, Vs, Ss = _buffers(probs, torch.float32)
    b = qlr.Batch(ctx, As, [P.k for P in probs], [P.p for P in probs], 3, Os, Us, Ss, Vs,
                  compute=qlr.COMPUTE_TF32X3, graph=False)
    assert not b.info()["graph"]
    for s in Ss:
        s.zero_()
    b.run()
    assert ctx.sync() == 0
    for i, P in enumerate(probs):
        ref = al.alg2_arbitrary_pass(P.A, P.k, P.p, 3, P.Omega)
        np.testing.assert_allclose(Ss[i].cpu().numpy(), ref.S, rtol=1e-4, err_msg=f"problem {i}")
    b.close()


def test_batch_plan_rejects_unaligned_pitch(ctx):
    """An unpadded BF16 row pitch (n not a multiple of 8) cannot feed TMA: the plan refuses, and
    the one-shot batched call falls back to the per-problem loop with the same answer."""
    from paper_2507_13731_gb300 import qlr
    probs = synth.batched_problems(count=3, seed=44, mmin=70, mmax=90, nmin=65, nmax=71, rmax=10)
    assert any(P.n % 8 for P in probs)
    As = [torch.from_numpy(np.ascontiguousarray(P.A[1:])).to(torch.bfloat16).cuda() for P in probs]
    Os = [dev_thin(P.Omega, "f32") for P in probs]
    Us = [qlr.empty_thin(P.m, P.k) for P in probs]
    Vs = [qlr.empty_thin(P.n, P.k) for P in probs]
    Ss = [torch.zeros(P.k, dtype=torch.float64, device="cuda") for P in probs]
    with pytest.raises(qlr.QlrError):
        qlr.Batch(ctx, As, [P.k for P in probs], [P.p for P in probs], 3, Os, Us, Ss, Vs)
    qlr.qsvd_lowrank_batched(ctx, As, [P.k for P in probs], [P.p for P in probs], 3, Os, Us, Ss, Vs)
    assert ctx.sync() == 0
    for i, P in enumerate(probs):
        ref = al.alg2_arbitrary_pass(P.A, P.k, P.p, 3, P.Omega)
        np.testing.assert_allclose(Ss[i].cpu().numpy(), ref.S, rtol=2e-2)


@pytest.mark.parametrize("variant", [2, 10, 15])
def test_batch_mixed_pure_and_full_quaternion(ctx, monkeypatch, variant):
    """A batch whose problems are partly full quaternion (a real plane present): the grouped
    sketch then stages all four A planes for every problem, in the plain and the fused-plane
    forms (variants 10 and 15: column blocks <= 64, one MMA per input plane); sigma against the
    oracle on the same matrices."""
    from paper_2507_13731_gb300 import qlr
    monkeypatch.setenv("QLR_BATCH_VARIANT", str(variant))
    probs = synth.batched_problems(count=40, seed=47, mmax=700, nmax=500, rmax=40)
    rng = np.random.default_rng(7)
    for i, P in enumerate(probs):
        if i % 2 == 0:   # a real plane at the noise level: the problem is no longer pure
            P.A[0] = 1e-3 * rng.standard_normal(P.A[0].shape)
            P.pure = False
    As, Os, Us, Vs, Ss = _buffers(probs, torch.bfloat16)
    b = qlr.Batch(ctx, As, [P.k for P in probs], [P.p for P in probs], 3, Os, Us, Ss, Vs, graph=False)
    assert ctx.sync() == 0 and b.info()["tile_order"] == variant
    for i in (0, 1, 20, 39):
        P = probs[i]
        ref = al.alg2_arbitrary_pass(P.A, P.k, P.p, 3, P.Omega)
        np.testing.assert_allclose(Ss[i].cpu().numpy(), ref.S, rtol=2e-2, err_msg=f"problem {i}")
        assert _orth_err(Us[i]) < 1e-4 and _orth_err(Vs[i]) < 1e-4
    b.close()
