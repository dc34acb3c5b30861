"""Degenerate sizes of the sketch product (eq. 1 summed over an inner index): an empty output
launches nothing and returns QLR_OK; an empty inner dimension is an empty sum, so Y = 0."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("compute,tdt", [("F64", torch.float64), ("F32", torch.float32),
                                         ("TF32X3", torch.float32)])
@pytest.mark.parametrize("op", ["N", "H"])
def test_sketch_empty_operands(compute, tdt, op):
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    ctx = qlr.Context(0)
    cm = getattr(qlr, "COMPUTE_" + compute)
    o = qlr.OP_N if op == "N" else qlr.OP_H
    # no output rows: A has no rows (op N) or no columns (op H)
    A = torch.zeros(4, 0, 6, dtype=tdt, device="cuda") if op == "N" else torch.zeros(4, 6, 0, dtype=tdt, device="cuda")
    X = qlr.empty_thin(6, 3, tdt)
    Y = qlr.empty_thin(0, 3, tdt)
    qlr.qsketch(ctx, o, A, X, Y, cm)
    # no output columns (l = 0)
    A = torch.ones(4, 5, 6, dtype=tdt, device="cuda")
    X = qlr.empty_thin(6 if op == "N" else 5, 0, tdt)
    Y = qlr.empty_thin(5 if op == "N" else 6, 0, tdt)
    qlr.qsketch(ctx, o, A, X, Y, cm)
    # empty inner dimension: Y = 0
    A = torch.zeros(4, 5, 0, dtype=tdt, device="cuda") if op == "N" else torch.zeros(4, 0, 5, dtype=tdt, device="cuda")
    X = qlr.empty_thin(0, 3, tdt)
    Y = qlr.empty_thin(5, 3, tdt)
    Y.fill_(float("nan"))
    qlr.qsketch(ctx, o, A, X, Y, cm)
    assert ctx.sync() == 0
    assert bool(torch.all(Y == 0))
    ctx.close()
