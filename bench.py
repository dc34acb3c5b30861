#!/usr/bin/env python3
"""Benchmark of the pass-efficient randomized quaternion QSVD on GB300 (one JSON line).

Workload (one "step"): the FP32 arbitrary-pass range finder workload -- a 4096 x 4096 quaternion
matrix with FP32 planes, sigma_i = 1/i and Haar-like singular vectors, k = 100, p = 10 -- run
through Algorithm 2 with each pass budget v in {2, 3, 4, 6, 8}: 23 sketch passes with their
orthonormalisations, five core QSVDs and lifts.  Metric: sketch passes per second (whole job);
A-read TB/s and the per-v rank-k QSVD times go in extra keys.  On one GPU the line also carries
`batched` (512 uneven BF16 problems as one batch plan against the plain FP32 per-problem loop),
`completion` (matrix completion's alternating updates on a 4096 x 4096 matrix with 70 % of the
entries removed, and the masked update kernel's roofline) and `lowrank_sweep` (the random rank-50
example at m = n = 500..4000); --no-batched / --no-completion / --no-sweep skip them.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank runs its own replica (weak scaling, no collective on the
data path); rank 0 prints the line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M = N = 4096
K_RANK, P_OVER = 100, 10
PASSES = (2, 3, 4, 6, 8)
METRIC = "sketch passes/s & A-read TB/s; rank-k QSVD time at stated error, BF16/batched vs FP32"
WORKLOAD = "slow-decay 4096x4096 quaternion, FP32 planes, sigma_i=1/i, k=100, p=10, Algorithm 2 at v in {2,3,4,6,8}"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=lambda: self.lines.extend(self.proc.stdout), daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_work(kid: str, compute: str):
    """(flops, bytes, bound, peak, unit, peak_note) per launch of a kernel class at this workload.
    Flops count 32 m n l per quaternion sketch (the Hamilton product, no split overhead)."""
    pk, src = _peaks()
    l = K_RANK + P_OVER
    sk_flops, sk_bytes = 32.0 * M * N * l, 4.0 * M * N * 4
    tf32 = pk.get("bf16_tflops_sustained", 1700.0) * (1.1 / 2.25)
    if kid == "sketch_tc":
        if compute == "BF16":
            return sk_flops, sk_bytes / 2, "tensor", pk.get("bf16_tflops_sustained", 1700.0), "TFLOP/s", \
                f"bf16 sustained ({src})"
        return sk_flops, sk_bytes, "tensor", tf32, "TFLOP/s", f"tf32 = bf16 sustained ({src}) x 1.1/2.25 nominal"
    fp32_simt = 152 * 128 * 2 * 2.07e9 / 1e12          # unit counts x max SM clock
    fp64 = 1.25                                         # nominal dense FP64 of the part
    if kid == "sketch_simt":
        return sk_flops, sk_bytes, "alu", fp32_simt, "TFLOP/s", "FP32 SIMT: 152 SMs x 128 lanes x 2 x 2.07 GHz"
    if kid == "gram":
        return 32.0 * M * l * (l + 1) / 2, 16.0 * M * l, "alu", fp64, "TFLOP/s", "FP64 nominal 1.25 TFLOP/s"
    if kid == "chol":
        return 32.0 * l ** 3 / 6, 32.0 * l * l, "alu", fp64, "TFLOP/s", "FP64 nominal 1.25 TFLOP/s"
    if kid == "tri_inv":
        return 32.0 * l ** 3 / 6, 32.0 * l * l, "alu", fp64, "TFLOP/s", "FP64 nominal 1.25 TFLOP/s"
    if kid == "jacobi":
        return 8 * 56.0 * l ** 3 / 2, 32.0 * l * l, "alu", fp32_simt, "TFLOP/s", "FP32 SIMT peak (one CTA can reach 1/152 of it)"
    return None


def roofline(stats, compute, steps):
    live = {k: v for k, v in stats.items() if v[0] > 0}
    dom = max(live, key=lambda k: live[k][1])
    n, ms = live[dom]
    w = algorithmic_work(dom, compute)
    out = {"kernel": dom, "launches": n, "avg_ms": ms / n}
    if w is None:
        out.update({"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None})
        return out
    flops, nbytes, bound, peak, unit, note = w
    sec = ms / n / 1e3
    if bound == "hbm":
        ach = nbytes / sec / 1e9
    else:
        ach = flops / sec / 1e12
    traffic = None
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        ent = tr.get(dom)
        if ent and ent.get("source_sha") == _source_sha(ent.get("source", "")):
            traffic = ent.get("dram_bytes_per_launch")
    except Exception:
        pass
    out.update({"bound": bound, "achieved": round(ach, 3), "peak": round(peak, 3), "unit": unit,
                "frac": round(ach / peak, 4), "traffic": traffic, "peak_source": note,
                "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": nbytes})
    return out


def _source_sha(rel):
    import hashlib
    p = os.path.join(ROOT, rel)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16] if rel and os.path.exists(p) else None


def cpu_oracle_sample(P, passes=2):
    """The FP64 oracle, as it stands, on a bounded sample of the workload: Algorithm 2 with v=2 on
    the full matrix.  Returns (passes/s, seconds, threads)."""
    from oracle import algorithms as al
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t0 = time.perf_counter()
    al.alg2_arbitrary_pass(P.A, P.k, P.p, passes, P.Omega)
    dt = time.perf_counter() - t0
    return passes / dt, dt, threads


BATCH_WORKLOAD = ("512 pure quaternion matrices, m ~ U{64..1024}, n ~ U{64..768}, rank r ~ U{8..64} plus "
                  "N(0,(1e-3)^2) noise on the i,j,k planes, k=r, p=8, Algorithm 2 with v=3, BF16 storage (16-byte row pitch)")


def batched_leg(dev, steps=5):
    """The batched workload: one batch plan (grouped tensor-core sketch per pass, per-problem
    orthonormalisation lanes, CUDA graph, tile-order autotuner) against the plain FP32 comparator,
    a loop of per-problem calls with FP32 storage and the FP32 SIMT sketch."""
    import numpy as np
    import torch

    import synth
    from paper_2507_13731_gb300 import qlr
    probs = synth.batched_problems()
    ctx = qlr.Context(dev.index or 0)
    As, Af = [], []
    for P in probs:
        t = qlr.empty_rowmajor(P.m, P.n, 3, torch.bfloat16, device=dev)
        src = torch.from_numpy(np.ascontiguousarray(P.A[1:]))
        t.copy_(src.to(torch.bfloat16))
        As.append(t)
        Af.append(src.float().to(dev))
    Os = [qlr.to_thin(torch.from_numpy(P.Omega).float().to(dev)) for P in probs]
    Us = [qlr.empty_thin(P.m, P.k, device=dev) for P in probs]
    Vs = [qlr.empty_thin(P.n, P.k, device=dev) for P in probs]
    Ss = [torch.zeros(P.k, dtype=torch.float64, device=dev) for P in probs]
    ks, ps = [P.k for P in probs], [P.p for P in probs]
    b = qlr.Batch(ctx, As, ks, ps, 3, Os, Us, Ss, Vs)
    info = b.info()
    for _ in range(3):
        b.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        b.run()
    e1.record()
    torch.cuda.synchronize()
    plan_ms = e0.elapsed_time(e1) / steps
    rc = ctx.sync()
    qlr.qsvd_lowrank_batched(ctx, Af, ks, ps, 3, Os, Us, Ss, Vs, compute=qlr.COMPUTE_F32)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(2):
        qlr.qsvd_lowrank_batched(ctx, Af, ks, ps, 3, Os, Us, Ss, Vs, compute=qlr.COMPUTE_F32)
    e1.record()
    torch.cuda.synchronize()
    loop_ms = e0.elapsed_time(e1) / 2
    rc = rc or ctx.sync()
    pk, src = _peaks()
    a_bytes = sum(3 * P.m * P.n * 2 for P in probs)
    pass_ms = info["tune_ms"][info["tile_order"]] / 2
    hbm = a_bytes / (pass_ms / 1e3) / 1e9
    b.close()
    ctx.close()
    return {"workload": BATCH_WORKLOAD, "plan_ms": round(plan_ms, 3),
            "problems_per_s": round(len(probs) / (plan_ms / 1e3), 1), "loop_fp32_ms": round(loop_ms, 3),
            "speedup_vs_fp32_loop": round(loop_ms / plan_ms, 2),
            "grouped_sketch": {"ms_per_pass": round(pass_ms, 4), "a_bytes_per_pass": a_bytes,
                               "hbm_gbs": round(hbm, 1), "peak_gbs": pk.get("hbm_gbs"),
                               "frac": round(hbm / pk.get("hbm_gbs", 6800.0), 4), "peak_source": src},
            "graph": info["graph"], "lanes": info["lanes"], "tile_order": info["tile_order"],
            "autotune_ms": [round(x, 4) for x in info["tune_ms"]], "launches_per_run": info["launches_per_run"],
            "device_error": rc}


COMPLETE_M = COMPLETE_N = 4096
COMPLETE_K, COMPLETE_P, COMPLETE_ITERS = 30, 10, 20
COMPLETE_WORKLOAD = ("matrix completion: 4096x4096 pure quaternion matrix of rank 30 plus N(0,(1e-2)^2) noise on the "
                     "i,j,k planes, FP32 planes, 70% of the entries removed uniformly at random, k=30, p=10, "
                     "Algorithm 2 with v=2 per iteration, 20 alternating updates from P_Omega(M) (the paper's colour "
                     "images with 70% of the pixels removed, R=30, two passes, scaled up)")


def completion_problem():
    import synth
    return synth.completion_problem(COMPLETE_M, COMPLETE_N, COMPLETE_K, missing=0.7, seed=1240, noise=1e-2,
                                    k=COMPLETE_K, p=COMPLETE_P)


def completion_leg(dev, steps=5):
    """Matrix completion (Section 7): one qlr_qcomplete call of COMPLETE_ITERS alternating updates
    (after one warm-up call), the masked update kernel alone (`steps` launches; M and C together
    exceed L2) and the completed matrix's error on the removed entries."""
    import numpy as np
    import torch

    from paper_2507_13731_gb300 import qlr
    P = completion_problem()
    m, n, k = P.m, P.n, P.k
    ctx = qlr.Context(dev.index or 0)
    mask = torch.from_numpy(P.extra["mask"]).to(dev)
    Md = torch.from_numpy(np.ascontiguousarray(P.A[1:])).float().to(dev)
    Cd = torch.empty(4, m, n, dtype=torch.float32, device=dev)
    Ud, Vd = qlr.empty_thin(m, k, device=dev), qlr.empty_thin(n, k, device=dev)
    Sd = torch.zeros(k, dtype=torch.float64, device=dev)
    Od = qlr.to_thin(torch.from_numpy(P.Omega).float().to(dev))
    qlr.complete(ctx, Md, mask, k, P.p, 2, 1, Od, Cd, Ud, Sd, Vd)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    qlr.complete(ctx, Md, mask, k, P.p, 2, COMPLETE_ITERS, Od, Cd, Ud, Sd, Vd)
    e1.record()
    torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    rc = ctx.sync()
    miss = P.extra["mask"] == 0
    C = Cd.cpu().double().numpy()
    err = float(np.sqrt(((C - P.A)[:, miss] ** 2).sum() / (P.A[:, miss] ** 2).sum()))
    for _ in range(3):
        qlr.complete_update(ctx, Md, mask, Cd, Ud, Sd, Vd, k)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        qlr.complete_update(ctx, Md, mask, Cd, Ud, Sd, Vd, k)
    e1.record()
    torch.cuda.synchronize()
    up_ms = e0.elapsed_time(e1) / steps
    rc = rc or ctx.sync()
    ctx.close()
    flops = 32.0 * m * n * k
    obs = float(P.extra["mask"].mean())
    nbytes = m * n * (1 + 16 + 12 * obs)           # mask, C written, M read at observed entries
    peak = 152 * 128 * 2 * 2.07e9 / 1e12
    ach = flops / (up_ms / 1e3) / 1e12
    return {"workload": COMPLETE_WORKLOAD, "iters": COMPLETE_ITERS, "ms_total": round(total_ms, 3),
            "ms_per_iter": round(total_ms / COMPLETE_ITERS, 3), "unobserved_rel_err": round(err, 6),
            "update_kernel": {"ms": round(up_ms, 4), "bound": "alu", "achieved": round(ach, 3), "peak": round(peak, 3),
                              "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                              "peak_source": "FP32 SIMT: 152 SMs x 128 lanes x 2 x 2.07 GHz",
                              "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": nbytes,
                              "hbm_gbs": round(nbytes / (up_ms / 1e3) / 1e9, 1)},
            "device_error": rc}


SWEEP_SIZES = tuple(range(500, 4001, 500))
SWEEP_CASES = (("alg2", 2), ("alg2", 3), ("alg1", 4), ("alg1", 6))
SWEEP_WORKLOAD = ("random low-rank example: A = B C with Gaussian quaternion B (m x 50) and C (50 x n), m = n = "
                  "500..4000 step 500, FP32 planes, k = 50, p = 10, Algorithm 2 with v = 2, 3 and Algorithm 1 with "
                  "q = 1, 2 (v = 4, 6)")


def lowrank_sweep_leg(dev, reps=3):
    """The random low-rank example of the experiments (Section 8): per size and algorithm the mean
    time of `reps` qlr_qsvd_lowrank calls (after one warm-up call) and the relative Frobenius error
    ||A - U S V^H||_F / ||A||_F (U S V^H formed by qlr_qcomplete_update with no observed entry)."""
    import torch

    import synth
    from paper_2507_13731_gb300 import qlr
    ctx = qlr.Context(dev.index or 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for m in SWEEP_SIZES:
        P = synth.random_lowrank_problem(m, m, 50)
        A = torch.from_numpy(P.A).float().to(dev).contiguous()
        om = qlr.to_thin(torch.from_numpy(P.Omega).float().to(dev))
        U, V = qlr.empty_thin(m, P.k, device=dev), qlr.empty_thin(m, P.k, device=dev)
        S = torch.zeros(P.k, dtype=torch.float64, device=dev)
        X = torch.empty_like(A)
        none = torch.zeros(m, m, dtype=torch.uint8, device=dev)
        nrm = float(torch.linalg.vector_norm(A.double()))
        ent = {"m": m, "n": m}
        for algo, v in SWEEP_CASES:
            a = qlr.ALG1 if algo == "alg1" else qlr.ALG2
            for _ in range(reps + 1):
                if _ == 1:
                    e0.record()
                qlr.qsvd_lowrank(ctx, A, P.k, P.p, v, om, U, S, V, algo=a, side=qlr.SIDE_X)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            qlr.complete_update(ctx, A, none, X, U, S, V, P.k)
            err = float(torch.linalg.vector_norm((A - X).double())) / nrm
            name = f"alg2_v{v}" if algo == "alg2" else f"alg1_q{v // 2 - 1}"
            ent[name] = {"ms": round(ms, 3), "rel_err": float(f"{err:.3e}")}
        rows.append(ent)
    rc = ctx.sync()
    ctx.close()
    return {"workload": SWEEP_WORKLOAD, "results": rows, "device_error": rc}


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """The largest of the ranks' values (the whole job is as slow as its slowest replica)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ws: int, elapsed_ms: float) -> float:
    """Units processed by all replicas per second, timed by the slowest one."""
    return ws * units_per_rank / (elapsed_ms / 1e3)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def run_reference(args, ws, rank):
    """Reference arm: the FP64 CPU oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import synth
    P = synth.config2(2)
    for _ in range(args.warmup):
        cpu_oracle_sample(P)
    t0 = time.perf_counter()
    thr = 0
    for _ in range(args.steps):
        _, _, thr = cpu_oracle_sample(P)
    dt = time.perf_counter() - t0
    value = 2 * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "sketch passes/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "Algorithm 2, v=2, full 4096x4096 matrix per step"},
            "cpu_baseline": {"value": round(value, 5), "unit": "sketch passes/s", "cores": thr, "kind": "oracle",
                             "sample": "Algorithm 2 with v=2 on the full 4096x4096 matrix per step"},
            "e2e": {"value": round(value, 5), "unit": "sketch passes/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_driver(args):
    """--only batch: the batched workload's plan (built once), then `warmup + steps` runs;
    QLR_BATCH_VARIANT=0..3 fixes the grouped sketch variant.  One JSON line."""
    import numpy as np
    import torch

    import synth
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    probs = synth.batched_problems()
    ctx = qlr.Context(0)
    As = []
    for P in probs:
        t = qlr.empty_rowmajor(P.m, P.n, 3, torch.bfloat16)
        t.copy_(torch.from_numpy(np.ascontiguousarray(P.A[1:])).to(torch.bfloat16))
        As.append(t)
    Os = [qlr.to_thin(torch.from_numpy(P.Omega).float().cuda()) for P in probs]
    Us = [qlr.empty_thin(P.m, P.k) for P in probs]
    Vs = [qlr.empty_thin(P.n, P.k) for P in probs]
    Ss = [torch.zeros(P.k, dtype=torch.float64, device="cuda") for P in probs]
    b = qlr.Batch(ctx, As, [P.k for P in probs], [P.p for P in probs], 3, Os, Us, Ss, Vs)
    for _ in range(args.warmup):
        b.run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        b.run()
    e1.record()
    torch.cuda.synchronize()
    rc = ctx.sync()
    print(json.dumps({"only": "batch", "ms_per_run": e0.elapsed_time(e1) / args.steps, "info": b.info(),
                      "device_error": rc}), flush=True)
    b.close()
    ctx.close()
    return 0 if rc == 0 else 1


def complete_driver(args):
    """--only complete: the completion workload's masked update kernel, `warmup + steps` launches."""
    import numpy as np
    import torch

    from paper_2507_13731_gb300 import build, qlr
    build.build()
    P = completion_problem()
    m, n, k = P.m, P.n, P.k
    ctx = qlr.Context(0)
    mask = torch.from_numpy(P.extra["mask"]).cuda()
    Md = torch.from_numpy(np.ascontiguousarray(P.A[1:])).float().cuda()
    Cd = torch.empty(4, m, n, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(0)
    Ud = qlr.to_thin(torch.from_numpy(rng.standard_normal((4, m, k))).float().cuda())
    Vd = qlr.to_thin(torch.from_numpy(rng.standard_normal((4, n, k))).float().cuda())
    Sd = torch.ones(k, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        qlr.complete_update(ctx, Md, mask, Cd, Ud, Sd, Vd, k)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        qlr.complete_update(ctx, Md, mask, Cd, Ud, Sd, Vd, k)
    e1.record()
    torch.cuda.synchronize()
    rc = ctx.sync()
    print(json.dumps({"only": "complete", "ms_per_call": e0.elapsed_time(e1) / args.steps, "device_error": rc}),
          flush=True)
    ctx.close()
    return 0 if rc == 0 else 1


def profile_driver(args):
    """Small driver for ncu captures: the bench workload's A and Omega, then `warmup + steps`
    calls of one sketch pass (--only sketch --op N|H) or one QSVD with --passes v (--only qsvd).
    Prints one JSON line with the mean CUDA-event time of the timed calls."""
    import numpy as np
    import torch

    if args.only == "batch":
        return batch_driver(args)
    if args.only == "complete":
        return complete_driver(args)

    import synth
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    P = synth.config2(args.passes)
    compute = getattr(qlr, "COMPUTE_" + args.compute)
    a_dt = torch.bfloat16 if args.compute == "BF16" else torch.float32
    A = torch.from_numpy(P.A).to(a_dt).cuda().contiguous()
    om = qlr.to_thin(torch.from_numpy(P.Omega).float().cuda())
    ctx = qlr.Context(0)
    U, V = qlr.empty_thin(M, K_RANK), qlr.empty_thin(N, K_RANK)
    S = torch.zeros(K_RANK, dtype=torch.float64, device="cuda")
    Y = qlr.empty_thin(M, K_RANK + P_OVER)
    op = qlr.OP_N if args.op == "N" else qlr.OP_H

    def call():
        if args.only == "sketch":
            qlr.qsketch(ctx, op, A, om, Y, compute)
        else:
            qlr.qsvd_lowrank(ctx, A, K_RANK, P_OVER, args.passes, om, U, S, V, compute=compute, side=qlr.SIDE_X)

    for _ in range(args.warmup):
        call()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    rc = ctx.sync()
    print(json.dumps({"only": args.only, "op": args.op, "passes": args.passes, "compute": args.compute,
                      "ms_per_call": e0.elapsed_time(e1) / args.steps, "device_error": rc}), flush=True)
    ctx.close()
    return 0 if rc == 0 else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--compute", default="TF32X3", choices=["TF32X3", "F32", "BF16", "TF32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched (512-problem) leg")
    ap.add_argument("--no-completion", action="store_true", help="skip the matrix-completion leg")
    ap.add_argument("--no-sweep", action="store_true", help="skip the random low-rank size sweep")
    ap.add_argument("--only", choices=["sketch", "qsvd", "batch", "complete"], default=None,
                    help="profiling driver: time only sketch passes, single QSVDs or batch runs (for ncu captures)")
    ap.add_argument("--op", choices=["N", "H"], default="N")
    ap.add_argument("--passes", type=int, default=4)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.only:
        return profile_driver(args)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import numpy as np
    import torch

    import synth
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P = synth.config2(4)
    compute = getattr(qlr, "COMPUTE_" + args.compute)
    a_dt = torch.bfloat16 if args.compute == "BF16" else torch.float32
    A_host = torch.from_numpy(P.A).to(a_dt).contiguous().pin_memory()
    Om_host = torch.from_numpy(np.ascontiguousarray(P.Omega.transpose(0, 2, 1))).float().contiguous().pin_memory()
    A = A_host.to(dev, non_blocking=True)
    om_store = Om_host.to(dev, non_blocking=True)
    om = om_store.transpose(1, 2)                                    # column-major n x l view
    U = qlr.empty_thin(M, K_RANK, device=dev)
    V = qlr.empty_thin(N, K_RANK, device=dev)
    S = torch.zeros(len(PASSES), K_RANK, dtype=torch.float64, device=dev)
    ctx = qlr.Context(local)
    ctx.reserve(max(qlr.workspace_size(M, N, K_RANK, P_OVER, v, qlr.ALG2, compute) for v in PASSES))
    qsvd_ms = {v: [] for v in PASSES}
    ev = {v: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for v in PASSES}

    def step(record=False):
        for i, v in enumerate(PASSES):
            if record:
                ev[v][0].record()
            qlr.qsvd_lowrank(ctx, A, K_RANK, P_OVER, v, om, U, S[i], V, compute=compute, side=qlr.SIDE_X)
            if record:
                ev[v][1].record()

    for _ in range(args.warmup):
        step()
    rc = ctx.sync()
    if rc != 0:
        raise SystemExit(f"device error {rc} during warm-up")

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    clocks = ClockSampler(local)
    ctx.reset_stats()
    ctx.set_timing(True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0e.record()
    for s in range(args.steps):
        step(record=(s == args.steps - 1))
    t1e.record()
    torch.cuda.synchronize()
    for v in PASSES:
        qsvd_ms[v].append(ev[v][0].elapsed_time(ev[v][1]))
    barrier()
    clk = clocks.stop()
    ctx.set_timing(False)
    elapsed_ms = t0e.elapsed_time(t1e)
    stats = ctx.stats()
    rc = ctx.sync()
    elapsed_ms = max_over_ranks(elapsed_ms, ws, dev)
    passes_per_step = sum(PASSES)
    value = whole_job_rate(passes_per_step * args.steps, ws, elapsed_ms)
    a_bytes = A.numel() * A.element_size()
    tbs = ws * passes_per_step * args.steps * a_bytes / (elapsed_ms / 1e3) / 1e12
    gpu_launches = sum(n for n, _ in stats.values())

    # end to end through the C ABI with host buffers: H2D of A and Omega, D2H of U, S, V per step
    U_h = torch.empty(4, K_RANK, M, dtype=torch.float32).pin_memory()
    V_h = torch.empty(4, K_RANK, N, dtype=torch.float32).pin_memory()
    S_h = torch.empty(len(PASSES), K_RANK, dtype=torch.float64).pin_memory()
    e2e_steps = max(2, min(args.steps, 3))
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(e2e_steps):
        A.copy_(A_host, non_blocking=True)
        om_store.copy_(Om_host, non_blocking=True)
        step()
        U_h.copy_(U.transpose(1, 2), non_blocking=True)
        V_h.copy_(V.transpose(1, 2), non_blocking=True)
        S_h.copy_(S, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, ws, dev)
    e2e_value = whole_job_rate(passes_per_step * e2e_steps, ws, e2e_ms)
    h2d = A_host.numel() * A_host.element_size() + Om_host.numel() * Om_host.element_size()
    d2h = U_h.numel() * 4 + V_h.numel() * 4 + S_h.numel() * 8

    line = None
    if rank == 0:
        roof = roofline(stats, args.compute, args.steps)
        cpu = None
        batched = None
        if ws == 1 and not args.no_batched:
            batched = batched_leg(dev)
        completion = None
        if ws == 1 and not args.no_completion:
            try:
                completion = completion_leg(dev)
            except Exception as e:                 # reported, never fatal to the headline line
                completion = {"error": f"{type(e).__name__}: {e}"}
        sweep = None
        if ws == 1 and not args.no_sweep:
            try:
                sweep = lowrank_sweep_leg(dev)
            except Exception as e:                 # reported, never fatal to the headline line
                sweep = {"error": f"{type(e).__name__}: {e}"}
        if ws == 1 and not args.no_cpu_baseline:
            val, secs, thr = cpu_oracle_sample(P)
            cpu = {"value": round(val, 5), "unit": "sketch passes/s", "cores": thr, "kind": "oracle",
                   "sample": f"Algorithm 2 with v=2 on the full 4096x4096 matrix ({secs:.1f} s)"}
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "sketch passes/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"TF32X3": "f32 (3xTF32 tensor-core sketch; FP64-class Gram (exact BF16 slices on tensor cores) "
                                "and Cholesky (double-FP32))", "F32": "f32 (SIMT)",
                      "BF16": "bf16 (FP32 accumulate; FP64-class Gram and Cholesky)", "TF32": "tf32"}[args.compute],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "passes": list(PASSES), "compute": args.compute,
                       "l2": "inputs larger than L2 (A = %.0f MB)" % (a_bytes / 1e6), "parallelism": f"replicas x{ws}"},
            "a_read_tbs": round(tbs, 4),
            "qsvd_ms": {str(v): round(statistics.mean(qsvd_ms[v]), 3) for v in PASSES},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_value, 3), "unit": "sketch passes/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": gpu_launches,
            "batched": batched,
            "completion": completion,
            "lowrank_sweep": sweep,
            "kernels": {k: {"launches": n, "ms": round(ms, 3)} for k, (n, ms) in stats.items() if n},
            "clocks": clk,
            "device_error": rc,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    ctx.close()


if __name__ == "__main__":
    main()
