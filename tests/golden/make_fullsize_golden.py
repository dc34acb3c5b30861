"""Writes tests/golden/fullsize_oracle.json: the FP64 oracle's results on the full-size seeded
workloads, against which the GPU tests and the benchmark state their errors.

Calls only the oracle (oracle/algorithms.py, oracle/norms.py) on the inputs of synth/ (seeded,
no method arithmetic).  For each workload and pass budget it stores the oracle's top-k singular
values and the two projection errors the error bounds of Section 4 govern -- the range error
||A - Q1 Q1^H A||_2 and the co-range error ||A - A Q2 Q2^H||_2 (Lemma 1, Theorem 3, eqs.
(mn11)/(mn12); Theorem 6 for Algorithm 4) -- with Q1, Q2 the oracle's final bases.

  python tests/golden/make_fullsize_golden.py [c2] [c3] [c4] [completion]   (default: all; about an hour)
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import algorithms as al  # noqa: E402
from oracle import completion as oc  # noqa: E402
from oracle import norms  # noqa: E402

OUT = os.path.join(HERE, "fullsize_oracle.json")


def entry(P, res, seconds):
    t = time.time()
    rng_err = norms.range_error(P.A, res.Q1)
    co_err = norms.corange_error(P.A, res.Q2)
    return {"k": P.k, "p": P.p, "sigma": [float(x) for x in res.S], "range_err": float(rng_err),
            "corange_err": float(co_err), "passes": res.passes, "columns": res.columns,
            "oracle_seconds": round(seconds, 1), "norm_seconds": round(time.time() - t, 1)}


def c2():
    out = {"workload": "4096x4096 quaternion, sigma_i = 1/i, Haar-like vectors (synth.config2), k=100, p=10, "
                       "Algorithm 2", "algo": 2}
    P = synth.config2(2)
    for v in (2, 3, 4, 6, 8):
        t = time.time()
        res = al.alg2_arbitrary_pass(P.A, P.k, P.p, v, P.Omega)
        out[f"v{v}"] = entry(P, res, time.time() - t)
        print("c2 v", v, out[f"v{v}"]["range_err"], out[f"v{v}"]["corange_err"], flush=True)
    return out


def c3():
    P = synth.config3()
    t = time.time()
    res = al.alg2_arbitrary_pass(P.A, P.k, P.p, 4, P.Omega)
    out = {"workload": "16384x8192 quaternion, sigma_i = exp(-i/50), Haar-like vectors (synth.config3), k=200, "
                       "p=20, Algorithm 2", "algo": 2, "v4": entry(P, res, time.time() - t)}
    print("c3", out["v4"]["range_err"], out["v4"]["corange_err"], flush=True)
    return out


def c4():
    P = synth.config4()
    t = time.time()
    res = al.alg4_block_flexible(P.A, P.k, P.p, 6, P.Omega)
    out = {"workload": "20000x10000 pure quaternion colour field (synth.config4), k=50, b=60, Algorithm 4",
           "algo": 4, "v6": entry(P, res, time.time() - t)}
    print("c4", out["v6"]["range_err"], out["v6"]["corange_err"], flush=True)
    return out


def completion():
    """Matrix completion (Section 7) at the benchmark's parameters: 4096 x 4096 rank-30 pure matrix
    plus noise 1e-2, 70 % removed, k = 30, p = 10, 20 alternating updates with 2 and 4 passes per
    update: the relative error on the removed entries and the last update's singular values."""
    P = synth.completion_problem(4096, 4096, 30, missing=0.7, seed=1240, noise=1e-2, k=30, p=10)
    miss = P.extra["mask"] == 0
    ref = float(np.sqrt((P.A[:, miss] ** 2).sum()))
    out = {"workload": "completion_problem(4096, 4096, 30, missing=0.7, seed=1240, noise=1e-2, k=30, p=10), "
                       "20 updates, Algorithm 2, side X"}
    for v in (2, 4):
        t = time.time()
        C, _, S, _, _ = oc.complete(P.A, P.extra["mask"], P.k, P.p, v, 20, P.Omega, side="X")
        err = float(np.sqrt(((C - P.A)[:, miss] ** 2).sum())) / ref
        out[f"v{v}"] = {"unobserved_rel_err": err, "sigma": [float(x) for x in S],
                        "oracle_seconds": round(time.time() - t, 1)}
        print("completion v", v, err, flush=True)
    return out


def main():
    which = sys.argv[1:] or ["c2", "c3", "c4", "completion"]
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data["citation"] = ("FP64 oracle results (oracle/algorithms.py Algorithms 2 and 4, oracle/norms.py spectral "
                        "norms by Lanczos on the complex adjoint) on the seeded full-size workloads of synth/, written "
                        "by tests/golden/make_fullsize_golden.py; Omega is each workload's seeded Gaussian test "
                        "matrix (Def. 2), side X.")
    for name in which:
        data[name] = {"c2": c2, "c3": c3, "c4": c4, "completion": completion}[name]()
        json.dump(data, open(OUT, "w"), indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
