"""Host logic of bench.py on CPU: the algorithmic work of sketch passes, the roofline object's
arithmetic and bound, the traffic figure's provenance check and the error statement."""
import json
import os

import numpy as np
import pytest

import bench


def test_sketch_work_counts_hamilton_flops_and_planes():
    f, b = bench.sketch_work(100, 80, [10, 30], pure=False, esz=4)
    assert f == 32.0 * 100 * 80 * 40 and b == 2 * 4 * 100 * 80 * 4
    f, b = bench.sketch_work(100, 80, [10], pure=True, esz=2)
    assert f == 24.0 * 100 * 80 * 10 and b == 3 * 100 * 80 * 2


def test_roofline_bound_and_fraction():
    pk, _ = bench._peaks()
    # narrow BF16 passes: A's bytes take longer than the flops at the BF16 rate -> HBM bound
    f, b = bench.sketch_work(20000, 10000, [8] * 4, pure=True, esz=2)
    r = bench.sketch_roofline(f, b, 4.0, 4, "BF16")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(b / 4e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / pk["hbm_gbs"], rel=1e-3)
    # wide 3xTF32 passes: three products per flop -> tensor bound, with the ceiling at a third
    f, b = bench.sketch_work(4096, 4096, [110] * 10, pure=False, esz=4)
    r = bench.sketch_roofline(f, b, 3.2, 10, "TF32X3")
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(f / 3.2e-3 / 1e12, rel=1e-3)
    assert r["frac_of_own_ceiling"] == pytest.approx(3 * r["frac"], rel=1e-3)
    assert r["algorithmic_flops_per_launch"] == pytest.approx(f / 10)


def test_traffic_only_for_the_measured_source():
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    tr = json.load(open(path)) if os.path.exists(path) else {}
    for key, ent in tr.items():
        if bench._source_sha(ent["source"]) == ent["source_sha"]:
            assert bench.traffic_for(key) == ent["dram_bytes_per_launch"]
        else:
            assert bench.traffic_for(key) is None
    assert bench.traffic_for("no_such_kernel") is None
    assert bench._source_sha("no/such/file.cu") is None


def test_sigma_error_statement():
    ref = np.array([4.0, 2.0, 1.0])
    assert bench.sigma_rel_err([4.0, 2.0, 1.0], ref) == 0.0
    assert bench.sigma_rel_err([4.0, 2.002, 0.999, 7.0], ref) == pytest.approx(1e-3)


def test_whole_job_rate_and_single_rank_max():
    assert bench.whole_job_rate(115, 2, 1000.0) == pytest.approx(230.0)
    assert bench.max_over_ranks(7.0, 1) == 7.0


def test_sketch_classes_of_the_mixed_mode():
    w = [60, 60, 60, 60, 60, 180]
    assert bench.sketch_classes("MIXED", w) == [("sketch_tc", "TF32", w[:-1]), ("sketch_x3", "TF32X3", [180])]
    assert bench.sketch_classes("TF32_RN", w) == [("sketch_tc", "TF32", w[:-1]), ("sketch_rn", "TF32_RN", [180])]
    assert bench.sketch_classes("TF32X3", w) == [("sketch_x3", "TF32X3", w)]
    assert bench.sketch_classes("BF16", w) == [("sketch_tc", "BF16", w)]
    assert bench.sketch_classes("F32", w) == [("sketch_simt", "F32", w)]


@pytest.mark.parametrize("op", ["N", "H"])
def test_library_reference_expansion_is_the_hamilton_product(op):
    """The cuBLAS reference leg computes the sketch through the real expansion of the Hamilton
    product; on CPU tensors it must equal the oracle's quaternion product of a pure A (eq. 1
    summed over the inner index; op H with A^H of Section 2)."""
    torch = pytest.importorskip("torch")
    from oracle import quaternion as Q
    m, n, l = 9, 7, 4
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, m, n))
    Afull = np.concatenate([np.zeros((1, m, n)), A])
    X = rng.standard_normal((4, n if op == "N" else m, l))
    got = bench.expansion_product(torch.from_numpy(A), bench.real_expansion(torch.from_numpy(X), op), op)
    rows = m if op == "N" else n
    got = got.reshape(rows, 4, l).permute(1, 0, 2).numpy()
    want = Q.qmatmul(Afull if op == "N" else Q.qH(Afull), X)
    np.testing.assert_allclose(got, want, atol=1e-12)
