"""Host logic of bench.py on CPU: the roofline object's arithmetic and the traffic figure's
provenance check."""
import json
import os

import pytest

import bench


def test_roofline_of_the_dominant_class():
    stats = {"sketch_tc": (10, 3.2), "jacobi": (5, 2.0), "gram": (0, 0.0)}
    r = bench.roofline(stats, "TF32X3", 1)
    assert r["kernel"] == "sketch_tc" and r["launches"] == 10
    flops = 32.0 * bench.M * bench.N * (bench.K_RANK + bench.P_OVER)
    assert r["algorithmic_flops_per_launch"] == flops
    assert r["achieved"] == pytest.approx(flops / 0.32e-3 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"


def test_bf16_sketch_counts_half_the_bytes():
    f32 = bench.algorithmic_work("sketch_tc", "TF32X3")
    bf16 = bench.algorithmic_work("sketch_tc", "BF16")
    assert bf16[1] == f32[1] / 2 and bf16[0] == f32[0]


def test_traffic_only_for_the_measured_source():
    tr = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    ent = tr["sketch_tc"]
    r = bench.roofline({"sketch_tc": (1, 1.0)}, "TF32X3", 1)
    if bench._source_sha(ent["source"]) == ent["source_sha"]:
        assert r["traffic"] == ent["dram_bytes_per_launch"]
    else:
        assert r["traffic"] is None
    assert bench._source_sha("no/such/file.cu") is None


def test_whole_job_rate_and_single_rank_max():
    assert bench.whole_job_rate(115, 2, 1000.0) == pytest.approx(230.0)
    assert bench.max_over_ranks(7.0, 1) == 7.0
