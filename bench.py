#!/usr/bin/env python3
"""Benchmark of the pass-efficient randomized quaternion QSVD on GB300 (one JSON line).

Headline workload (one "step"): the pass-efficient block Krylov workload -- a 20000 x 10000 pure
quaternion colour field (FP32 planes; per colour plane a sum of 64 random 2-D cosines, min-max
scaled to [0, 1], plus uniform noise of amplitude 0.05) -- through Algorithm 4 with k = 50, block
size b = 60 and v = 6 views: six sketch passes (five of 60 columns, the last of 180), the deflated
Krylov stack and its QR, the core QSVD of the 180 x 180 factor and the lifts, in TF32 (one TF32
product for the Krylov blocks, one product of operands rounded to nearest TF32 with chunked FP32
sums for the final pass; --compute picks another arithmetic; the same call with a 3xTF32 final
pass is timed beside it as `fp32_final_pass`).  Metric: sketch passes
per second (whole job); extra keys: A-read TB/s, ms per QSVD and the result's error against the FP64
oracle (the oracle's values on the same seeded input are stored in tests/golden/fullsize_oracle.json
by tests/golden/make_fullsize_golden.py): the largest relative error of the top-k singular values
and the projection errors ||A - Q1 Q1^H A||_2, ||A - A Q2 Q2^H||_2 of the call's final bases
(estimated on the GPU by qlr_residual_norm, outside the timed region).

On one GPU the line also carries
  `peaks`       the measured dense rates of this GPU's tensor and CUDA cores (the roofline
                denominators other than HBM and BF16, which MEASURED_PEAKS.json holds);
  `mixed_precision` the 16384 x 8192 exponential-decay workload (k = 200, p = 20, v = 4, Algorithm 2)
                with BF16 storage against the same call in 3xTF32 and in plain FP32 (SIMT), each
                with its time and its error against the oracle, plus the BF16 sketch's roofline;
  `pass_sweep`  the 4096 x 4096 slow-decay workload through Algorithm 2 at v in {2, 3, 4, 6, 8};
  `library_reference` cuBLAS (torch.matmul) on the materialised real expansion of the headline's
                narrow pass, FP32 and TF32 (a library reference, not this library's path);
  `batched`, `completion`, `lowrank_sweep` as named (--no-batched / --no-completion / --no-sweep).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--compute MODE]

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

METRIC = "sketch passes/s & A-read TB/s; rank-k QSVD time at stated error, BF16/batched vs FP32"
# headline: the block Krylov workload
HM, HN, HK, HB, HV = 20000, 10000, 50, 60, 6
WORKLOAD = ("pure quaternion colour field 20000x10000 (64 random 2-D cosines per colour plane, min-max scaled, "
            "+U[-0.05,0.05] noise), FP32 planes, Algorithm 4, k=50, b=60, v=6 (5 passes of 60 columns + 1 of 180)")
# the mixed-precision workload
C3 = dict(m=16384, n=8192, k=200, p=20, v=4)
C3_WORKLOAD = "exp-decay 16384x8192 quaternion, sigma_i=exp(-i/50), Haar-like vectors, k=200, p=20, Algorithm 2, v=4"
# the pass sweep
M = N = 4096
K_RANK, P_OVER = 100, 10
PASSES = (2, 3, 4, 6, 8)
C2_WORKLOAD = "slow-decay 4096x4096 quaternion, FP32 planes, sigma_i=1/i, k=100, p=10, Algorithm 2 at v in {2,3,4,6,8}"
# probe-measured peaks of this run (filled by peaks_leg)
_MEASURED = {}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _golden():
    try:
        return json.load(open(os.path.join(ROOT, "tests", "golden", "fullsize_oracle.json")))
    except Exception:
        return {}


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


# ------------------------------------------------------------------------------------------
# roofline arithmetic (host logic, tested on CPU)
def sketch_work(m: int, n: int, widths, pure: bool, esz: int):
    """Algorithmic work of sketch passes over an m x n quaternion A: flops 32 m n l per pass (24 for a
    pure A: its real plane is zero), bytes = A read once per pass (4 or 3 planes of esz bytes)."""
    planes = 3 if pure else 4
    flops = sum((8.0 * planes) * m * n * l for l in widths)
    nbytes = float(len(widths)) * planes * m * n * esz
    return flops, nbytes


def peak_for(compute: str):
    """(peak, unit, products per algorithmic flop, source note) of a sketch's arithmetic."""
    pk, src = _peaks()
    if compute == "BF16":
        return pk.get("bf16_tflops", 1900.0), "TFLOP/s", 1, f"bf16 burst ({src}, MEASURED_PEAKS.json)"
    if compute in ("TF32", "TF32X3", "MIXED", "TF32_RN"):
        if "tf32_mma" in _MEASURED:
            return _MEASURED["tf32_mma"], "TFLOP/s", 3 if compute == "TF32X3" else 1, \
                "tf32 tcgen05 MMA loop measured in this run (qlr_peak_probe)"
        return pk.get("bf16_tflops", 1900.0) * 0.5, "TFLOP/s", 3 if compute == "TF32X3" else 1, \
            f"tf32 = bf16 burst ({src}) x 1/2 nominal ratio (probe not run)"
    if compute == "F32":
        if "fp32_fma" in _MEASURED:
            return _MEASURED["fp32_fma"], "TFLOP/s", 1, "FP32 FMA loop measured in this run (qlr_peak_probe)"
        return 152 * 128 * 2 * 2.07e9 / 1e12, "TFLOP/s", 1, "FP32 SIMT: 152 SMs x 128 lanes x 2 x 2.07 GHz (nominal)"
    return None, None, 1, None


def sketch_roofline(flops: float, nbytes: float, ms: float, launches: int, compute: str, traffic=None):
    """Roofline object of the sketch launches of a timed region: achieved = algorithmic work of all
    launches / their summed CUDA-event time; bound = the roof the work meets first."""
    pk, src = _peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    peak, unit, products, note = peak_for(compute)
    sec = ms / 1e3
    t_hbm = nbytes / (hbm * 1e9)
    t_ops = flops * products / (peak * 1e12) if peak else 0.0
    out = {"kernel": "sketch_tc" if compute != "F32" else "sketch_simt", "launches": launches,
           "avg_ms": round(ms / max(launches, 1), 5), "algorithmic_flops_per_launch": flops / max(launches, 1),
           "algorithmic_bytes_per_launch": nbytes / max(launches, 1), "traffic": traffic}
    if t_hbm >= t_ops:
        ach = nbytes / sec / 1e9
        out.update({"bound": "hbm", "achieved": round(ach, 2), "peak": round(hbm, 1), "unit": "GB/s",
                    "frac": round(ach / hbm, 4), "peak_source": f"HBM copy ({src}, MEASURED_PEAKS.json)"})
    else:
        ach = flops / sec / 1e12
        out.update({"bound": "alu" if compute == "F32" else "tensor", "achieved": round(ach, 3),
                    "peak": round(peak, 2), "unit": unit, "frac": round(ach / peak, 4), "peak_source": note})
    out["hbm_gbs"] = round(nbytes / sec / 1e9, 1)
    if products > 1:
        out["products_per_flop"] = products
        out["frac_of_own_ceiling"] = round(out["frac"] * products, 4) if out["bound"] != "hbm" else None
    return out


def sketch_classes(compute: str, widths):
    """(statistics class, arithmetic, pass widths) of the sketch launches of one step: the mixed
    modes run the Krylov blocks in TF32 and the last pass in 3xTF32 (MIXED) or rounded TF32
    (TF32_RN), each a class of its own."""
    if compute == "MIXED":
        return [("sketch_tc", "TF32", list(widths[:-1])), ("sketch_x3", "TF32X3", [widths[-1]])]
    if compute == "TF32_RN":
        return [("sketch_tc", "TF32", list(widths[:-1])), ("sketch_rn", "TF32_RN", [widths[-1]])]
    kid = {"F32": "sketch_simt", "TF32X3": "sketch_x3", "TF32_RN": "sketch_rn"}.get(compute, "sketch_tc")
    return [(kid, compute, list(widths))]


def traffic_for(key: str):
    """DRAM bytes per launch from profiles/traffic.json, only while the kernel's source is the one
    the counters were taken on."""
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        ent = tr.get(key)
        if ent and ent.get("source_sha") == _source_sha(ent.get("source", "")):
            return ent.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


def _source_sha(rel):
    import hashlib
    p = os.path.join(ROOT, rel)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16] if rel and os.path.exists(p) else None


def sigma_rel_err(S, ref) -> float:
    import numpy as np
    S, ref = np.asarray(S, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(S[:len(ref)] - ref) / ref))


# ------------------------------------------------------------------------------------------
def colour_problem():
    import synth
    return synth.config4()


def errors_vs_oracle(ctx, A, P, S, algo, v, compute, golden, side=0, iters=30, nvec=8):
    """The result's error statement: sigma relative error against the oracle's, and the projection
    errors of the call's final bases (qlr_qbasis, then qlr_residual_norm) beside the oracle's."""
    import torch

    import synth
    from paper_2507_13731_gb300 import qlr
    out = {}
    if golden and "sigma" in golden:
        out["sigma_rel_err"] = float(f"{sigma_rel_err(S, golden['sigma']):.3e}")
    l = P.k + P.p
    L = qlr.stacked_width(algo, l, v)
    om = qlr.to_thin(torch.from_numpy(P.Omega).float().to(A.device))
    Q1, Q2 = qlr.empty_thin(P.m, L, device=A.device), qlr.empty_thin(P.n, L, device=A.device)
    R = torch.zeros(4, L, L, dtype=torch.float64, device=A.device)
    qlr.qbasis(ctx, A, P.k, P.p, v, om, Q1, Q2, R, algo=algo, compute=compute, side=qlr.SIDE_X)
    start = qlr.to_thin(torch.from_numpy(synth.gaussian_qmat(4242, P.n, nvec)).float().to(A.device))
    e1 = qlr.residual_norm(ctx, A, Q1, qlr.SIDE_X, start, iters=iters)
    e2 = qlr.residual_norm(ctx, A, Q2, qlr.SIDE_XH, start, iters=iters)
    out["range_err"] = float(f"{e1:.6e}")
    out["corange_err"] = float(f"{e2:.6e}")
    if golden and "range_err" in golden:
        out["oracle_range_err"] = golden["range_err"]
        out["oracle_corange_err"] = golden["corange_err"]
        out["range_err_rel_diff"] = float(f"{abs(e1 - golden['range_err']) / golden['range_err']:.3e}")
        out["corange_err_rel_diff"] = float(f"{abs(e2 - golden['corange_err']) / golden['corange_err']:.3e}")
    out["estimator"] = f"block power iteration, {nvec} vectors, {iters} steps (a lower bound converging to the norm)"
    return out


def peaks_leg(dev):
    """Dense rates of this GPU measured by the library's probe kernels (qlr_peak_probe)."""
    from paper_2507_13731_gb300 import qlr
    d = dev.index or 0
    out = {}
    for name, kind in (("tf32_mma", qlr.PEAK_TF32_MMA), ("bf16_mma", qlr.PEAK_BF16_MMA),
                       ("fp32_fma", qlr.PEAK_FP32_FMA), ("fp64_fma", qlr.PEAK_FP64_FMA),
                       ("tf32_mma_n64", qlr.PEAK_TF32_MMA_N64), ("bf16_mma_n64", qlr.PEAK_BF16_MMA_N64)):
        try:
            out[name] = round(qlr.measure_peak(kind, d), 2)
        except Exception as e:                     # reported, never fatal to the headline line
            out[name] = None
            out[name + "_error"] = f"{type(e).__name__}: {e}"
    _MEASURED.update({k: v for k, v in out.items() if isinstance(v, float)})
    out["unit"] = "TFLOP/s"
    out["how"] = ("tcgen05 MMA loop, M=128 N=256 (K=8 tf32 / 16 bf16) from shared memory, one CTA per SM (the _n64 "
                  "entries: the same loop with N=64); FMA loops, 8 independent chains per thread, 8 CTAs of 256 threads "
                  "per SM; best of 3 ~40 ms launches")
    return out


# the Hamilton product's sign table: s(c, d) = -1 for these (input plane c, output plane d) of op N;
# op H flips every c != 0
_NEG_N = {(1, 0), (2, 0), (3, 0), (1, 2), (2, 3), (3, 1)}


def _hamilton_sign(c: int, d: int, op: str) -> float:
    s = -1.0 if (c, d) in _NEG_N else 1.0
    return -s if (op == "H" and c != 0) else s


def real_expansion(Xp, op: str):
    """The thin operand's side of the Hamilton product as a real matrix, for a pure A (planes
    1..3): per input plane c, the four output planes' blocks s(c, d) X_(c xor d) side by side.
    Xp: (4, rows, l) -> (3, rows, 4 l)."""
    import torch
    return torch.stack([torch.cat([_hamilton_sign(c, d, op) * Xp[c ^ d] for d in range(4)], dim=1)
                        for c in (1, 2, 3)])


def expansion_product(A, Ex, op: str):
    """The sketch product of a pure A (3, m, n) through the real expansion: op N as the batched
    product over the planes summed, op H as one product on the stacked planes.  Returns the four
    output planes side by side, (rows_out, 4 l)."""
    import torch
    if op == "N":
        return torch.matmul(A, Ex).sum(0)
    m, n = A.shape[1], A.shape[2]
    return torch.matmul(A.reshape(3 * m, n).t(), Ex.reshape(3 * m, Ex.shape[2]))


def library_leg(ctx, A, ell=HB, reps=5):
    """A library reference for the headline's narrow sketch pass (pure A, l = 60): cuBLAS through
    torch.matmul on the materialised real expansion of the Hamilton product, FP32 (TF32 off) and
    TF32 -- op N as Y_d = sum_c s(c, d) A_c X_(c xor d) (one batched product over the planes and a
    sum), op H as Z = [A_1; A_2; A_3]^T F(Y) (one product on the stacked planes).  Checked against
    this library's 3xTF32 product; not this library's path."""
    import torch

    from paper_2507_13731_gb300 import qlr
    dev = A.device
    m, n = A.shape[1], A.shape[2]
    g = torch.Generator(device=dev).manual_seed(7)
    out = {"workload": f"pure {m}x{n} FP32 planes, l = {ell}", "reps": reps}
    prev = torch.backends.cuda.matmul.allow_tf32
    try:
        for op in ("N", "H"):
            rows_in, rows_out = (n, m) if op == "N" else (m, n)
            Xp = torch.randn(4, rows_in, ell, device=dev, generator=g)
            Ex = real_expansion(Xp, op)                                          # E (op N) or F (op H)
            call = lambda: expansion_product(A, Ex, op)                          # (rows_out, 4 l)
            ref = qlr.empty_thin(rows_out, ell, device=dev)
            qlr.qsketch(ctx, qlr.OP_N if op == "N" else qlr.OP_H, A, qlr.to_thin(Xp), ref, qlr.COMPUTE_TF32X3)
            for mode, tf32 in (("fp32", False), ("tf32", True)):
                torch.backends.cuda.matmul.allow_tf32 = tf32
                for _ in range(2):
                    Y = call()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    Y = call()
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                got = Y.reshape(rows_out, 4, ell).permute(1, 0, 2)
                err = float((got - ref).abs().max() / ref.abs().max())
                out[f"op{op}_{mode}"] = {"ms": round(ms, 4), "a_read_tbs": round(3 * m * n * 4 / (ms / 1e3) / 1e12, 3),
                                         "max_rel_diff_vs_3xtf32": float(f"{err:.2e}")}
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def cpu_oracle_sample(P):
    """The FP64 oracle, as it stands, on a bounded sample of the headline workload: one view of
    Algorithm 4 (Y = X Omega and the QR of Y) on the full matrix.  Returns (passes/s, s, threads)."""
    from oracle import quaternion as Q
    from oracle.qr import qr
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t0 = time.perf_counter()
    qr(Q.qmatmul(P.A, P.Omega))
    dt = time.perf_counter() - t0
    return 1.0 / dt, dt, threads


def mixed_precision_leg(dev, golden, reps=3):
    """The 16384 x 8192 workload (Algorithm 2, v = 4) with BF16 storage against the same call in
    3xTF32 and in plain FP32 (SIMT) on FP32 storage: time per QSVD, error against the oracle and
    the sketch's roofline in each arithmetic."""
    import numpy as np
    import torch

    import synth
    from paper_2507_13731_gb300 import qlr
    P = synth.config3()
    ctx = qlr.Context(dev.index or 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    om = qlr.to_thin(torch.from_numpy(P.Omega).float().to(dev))
    U, V = qlr.empty_thin(P.m, P.k, device=dev), qlr.empty_thin(P.n, P.k, device=dev)
    S = torch.zeros(P.k, dtype=torch.float64, device=dev)
    gold = golden.get("c3", {}).get("v4")
    out = {"workload": C3_WORKLOAD}
    Af = torch.from_numpy(P.A).float().to(dev).contiguous()
    Ab = Af.to(torch.bfloat16).contiguous()
    for mode, Ad in (("BF16", Ab), ("TF32X3", Af), ("F32", Af)):
        comp = getattr(qlr, "COMPUTE_" + mode)
        n = 1 if mode == "F32" else reps
        qlr.qsvd_lowrank(ctx, Ad, P.k, P.p, 4, om, U, S, V, compute=comp, side=qlr.SIDE_X)
        torch.cuda.synchronize()
        ctx.reset_stats()
        ctx.set_timing(True)
        e0.record()
        for _ in range(n):
            qlr.qsvd_lowrank(ctx, Ad, P.k, P.p, 4, om, U, S, V, compute=comp, side=qlr.SIDE_X)
        e1.record()
        torch.cuda.synchronize()
        ctx.set_timing(False)
        ms = e0.elapsed_time(e1) / n
        st = ctx.stats()
        ent = {"ms_per_qsvd": round(ms, 3)}
        ent.update(errors_vs_oracle(ctx, Ad, P, S.cpu().numpy(), qlr.ALG2, 4, comp, gold))
        kid = {"F32": "sketch_simt", "TF32X3": "sketch_x3"}.get(mode, "sketch_tc")
        nl, kms = st[kid]
        if nl:
            fl, nb = sketch_work(P.m, P.n, [P.k + P.p] * 4 * n, False, 2 if mode == "BF16" else 4)
            ent["sketch"] = sketch_roofline(fl, nb, kms, nl, mode,
                                            traffic_for("sketch_tc_bf16_c3") if mode == "BF16" else None)
        ent["kernels_ms_per_qsvd"] = {k: round(t / n, 3) for k, (c, t) in st.items() if c}
        out[mode] = ent
    rc = ctx.sync()
    out["bf16_speedup_vs_fp32_simt"] = round(out["F32"]["ms_per_qsvd"] / out["BF16"]["ms_per_qsvd"], 2)
    out["tf32x3_speedup_vs_fp32_simt"] = round(out["F32"]["ms_per_qsvd"] / out["TF32X3"]["ms_per_qsvd"], 2)
    out["tolerance"] = {"BF16": 2e-2, "TF32X3": 1e-4, "F32": 1e-4}
    out["device_error"] = rc
    ctx.close()
    return out


def pass_sweep_leg(dev, golden, compute="TF32X3", reps=3):
    """The 4096 x 4096 slow-decay workload through Algorithm 2 at each pass budget: ms per QSVD and
    the singular values' error against the oracle."""
    import torch

    import synth
    from paper_2507_13731_gb300 import qlr
    P = synth.config2(2)
    ctx = qlr.Context(dev.index or 0)
    A = torch.from_numpy(P.A).float().to(dev).contiguous()
    om = qlr.to_thin(torch.from_numpy(P.Omega).float().to(dev))
    U, V = qlr.empty_thin(M, K_RANK, device=dev), qlr.empty_thin(N, K_RANK, device=dev)
    S = torch.zeros(K_RANK, dtype=torch.float64, device=dev)
    comp = getattr(qlr, "COMPUTE_" + compute)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": C2_WORKLOAD, "compute": compute}
    for v in PASSES:
        qlr.qsvd_lowrank(ctx, A, K_RANK, P_OVER, v, om, U, S, V, compute=comp, side=qlr.SIDE_X)
        e0.record()
        for _ in range(reps):
            qlr.qsvd_lowrank(ctx, A, K_RANK, P_OVER, v, om, U, S, V, compute=comp, side=qlr.SIDE_X)
        e1.record()
        torch.cuda.synchronize()
        ent = {"ms_per_qsvd": round(e0.elapsed_time(e1) / reps, 3)}
        gold = golden.get("c2", {}).get(f"v{v}")
        if gold:
            ent["sigma_rel_err"] = float(f"{sigma_rel_err(S.cpu().numpy(), gold['sigma']):.3e}")
        out[f"v{v}"] = ent
    out["device_error"] = ctx.sync()
    ctx.close()
    return out


BATCH_WORKLOAD = ("512 pure quaternion matrices, m ~ U{64..1024}, n ~ U{64..768}, rank r ~ U{8..64} plus "
                  "N(0,(1e-3)^2) noise on the i,j,k planes, k=r, p=8, Algorithm 2 with v=3, BF16 storage (16-byte row pitch)")


def batched_leg(dev, steps=5):
    """The batched workload: one batch plan (grouped tensor-core sketch per pass, grouped
    orthonormalisation and core QSVD launches, CUDA graph, autotuner) against the plain FP32
    comparator, a loop of per-problem calls with FP32 storage and the FP32 SIMT sketch."""
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
                     "Algorithm 2 with v=4 (and v=2) per update, 20 alternating updates from P_Omega(M) (the paper's "
                     "colour images with 70% of the pixels removed, R=30, scaled up)")


def completion_problem():
    import synth
    return synth.completion_problem(COMPLETE_M, COMPLETE_N, COMPLETE_K, missing=0.7, seed=1240, noise=1e-2,
                                    k=COMPLETE_K, p=COMPLETE_P)


def completion_leg(dev, golden, steps=5):
    """Matrix completion (Section 7): one qlr_qcomplete call of COMPLETE_ITERS alternating updates
    per pass budget (after one warm-up call), the error on the removed entries beside the oracle's
    (stored values; with two passes per update the oracle itself stalls, with four it converges),
    and the masked update kernel alone (`steps` launches; M and C together exceed L2)."""
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
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    miss = P.extra["mask"] == 0
    ref = float(np.sqrt((P.A[:, miss] ** 2).sum()))
    out = {"workload": COMPLETE_WORKLOAD, "iters": COMPLETE_ITERS}
    rc = 0
    for v in (4, 2):
        qlr.complete(ctx, Md, mask, k, P.p, v, 1, Od, Cd, Ud, Sd, Vd)
        torch.cuda.synchronize()
        e0.record()
        qlr.complete(ctx, Md, mask, k, P.p, v, COMPLETE_ITERS, Od, Cd, Ud, Sd, Vd)
        e1.record()
        torch.cuda.synchronize()
        total_ms = e0.elapsed_time(e1)
        rc = rc or ctx.sync()
        C = Cd.cpu().double().numpy()
        err = float(np.sqrt(((C - P.A)[:, miss] ** 2).sum())) / ref
        ent = {"ms_total": round(total_ms, 3), "ms_per_iter": round(total_ms / COMPLETE_ITERS, 3),
               "unobserved_rel_err": round(err, 6)}
        gold = golden.get("completion", {}).get(f"v{v}")
        if gold:
            ent["oracle_unobserved_rel_err"] = round(gold["unobserved_rel_err"], 6)
            ent["sigma_rel_err"] = float(f"{sigma_rel_err(Sd.cpu().numpy(), gold['sigma']):.3e}")
        out[f"v{v}"] = ent
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
    peak, unit, _, note = peak_for("F32")
    ach = flops / (up_ms / 1e3) / 1e12
    out["update_kernel"] = {"ms": round(up_ms, 4), "bound": "alu", "achieved": round(ach, 3), "peak": round(peak, 3),
                            "unit": "TFLOP/s", "frac": round(ach / peak, 4), "peak_source": note,
                            "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": nbytes,
                            "hbm_gbs": round(nbytes / (up_ms / 1e3) / 1e9, 1)}
    out["device_error"] = rc
    return out


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
    """Reference arm: the FP64 CPU oracle timed on the host cores (rank 0 only), each step one view
    of Algorithm 4 on the headline matrix."""
    if rank != 0:
        return
    P = colour_problem()
    for _ in range(args.warmup):
        cpu_oracle_sample(P)
    t0 = time.perf_counter()
    thr = 0
    for _ in range(args.steps):
        _, _, thr = cpu_oracle_sample(P)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    sample = "one view of Algorithm 4 per step: Y = X Omega (60 columns) and the Householder QR of Y, full 20000x10000 matrix"
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "sketch passes/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": round(value, 5), "unit": "sketch passes/s", "cores": thr, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 5), "unit": "sketch passes/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
def profile_driver(args):
    """Small driver for ncu captures and probes: the named workload's A and Omega, then
    `warmup + steps` calls of one sketch pass (--only sketch --op N|H --ell L) or one QSVD
    (--only qsvd), or a batch plan (--only batch), or the completion update (--only complete), or
    the peak probes (--only peaks).  Prints one JSON line with the mean CUDA-event time."""
    import numpy as np
    import torch

    if args.only == "batch":
        return batch_driver(args)
    if args.only == "complete":
        return complete_driver(args)
    import synth
    from paper_2507_13731_gb300 import build, qlr
    build.build()
    if args.only == "peaks":
        print(json.dumps({"only": "peaks", "peaks": peaks_leg(torch.device("cuda", 0))}), flush=True)
        return 0
    compute = getattr(qlr, "COMPUTE_" + args.compute)
    a_dt = torch.bfloat16 if args.compute == "BF16" else torch.float32
    if args.m and args.n:          # a uniform pure matrix of the given size (small profiling cases)
        P, algo, v = synth.config_colour(max(args.m, 256), max(args.n, 256), HK, HB, HV), qlr.ALG4, HV
        g = torch.Generator(device="cuda").manual_seed(5)
        A = torch.rand(3, args.m, args.n, device="cuda", generator=g).to(a_dt).contiguous()
        P.A = P.A[:, :args.m, :args.n]
        P.Omega = P.Omega[:, :args.n, :]
    elif args.config == "c4":
        P, algo, v = colour_problem(), qlr.ALG4, HV
        A = torch.from_numpy(np.ascontiguousarray(P.A[1:])).to(a_dt).cuda().contiguous()
    elif args.config == "c3":
        P, algo, v = synth.config3(), qlr.ALG2, 4
        A = torch.from_numpy(P.A).to(a_dt).cuda().contiguous()
    else:
        P, algo, v = synth.config2(args.passes), qlr.ALG2, args.passes
        A = torch.from_numpy(P.A).to(a_dt).cuda().contiguous()
    m, n = P.m, P.n
    ell = args.ell or (P.k + P.p)
    ctx = qlr.Context(0)
    U, V = qlr.empty_thin(m, P.k), qlr.empty_thin(n, P.k)
    S = torch.zeros(P.k, dtype=torch.float64, device="cuda")
    om = qlr.to_thin(torch.from_numpy(P.Omega).float().cuda())
    op = qlr.OP_N if args.op == "N" else qlr.OP_H
    X = qlr.to_thin(torch.randn(4, n if op == qlr.OP_N else m, ell).cuda())
    Y = qlr.empty_thin(m if op == qlr.OP_N else n, ell)

    def call():
        if args.only == "sketch" and args.noalloc:
            qlr.qsketch_noalloc(op, A, X, Y, compute)
        elif args.only == "sketch":
            qlr.qsketch(ctx, op, A, X, Y, compute)
        else:
            qlr.qsvd_lowrank(ctx, A, P.k, P.p, v, om, U, S, V, algo=algo, compute=compute, side=qlr.SIDE_X)

    for _ in range(args.warmup):
        call()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    rc = ctx.sync()
    ms = e0.elapsed_time(e1) / args.steps
    # the same calls again with every kernel class bracketed by events (launches ms per call)
    ctx.reset_stats()
    ctx.set_timing(True)
    for _ in range(args.steps):
        call()
    st = ctx.stats()
    ctx.set_timing(False)
    rc = rc or ctx.sync()
    classes = {k: [round(nl / args.steps, 1), round(t / args.steps, 4)] for k, (nl, t) in st.items() if nl}
    print(json.dumps({"only": args.only, "config": args.config, "op": args.op, "ell": ell, "passes": v,
                      "compute": args.compute, "noalloc": bool(args.noalloc), "ms_per_call": ms,
                      "classes_launches_ms": classes,
                      "device_error": rc}), flush=True)
    ctx.close()
    return 0 if rc == 0 else 1


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
    graph_ms = e0.elapsed_time(e1) / args.steps
    info = b.info()
    b.close()
    # the same plan run eagerly, each kernel class timed with events on the context stream
    b = qlr.Batch(ctx, As, [P.k for P in probs], [P.p for P in probs], 3, Os, Us, Ss, Vs, graph=False)
    for _ in range(args.warmup):
        b.run()
    torch.cuda.synchronize()
    ctx.reset_stats()
    ctx.set_timing(True)
    for _ in range(args.steps):
        b.run()
    st = ctx.stats()
    ctx.set_timing(False)
    rc = rc or ctx.sync()
    per_run = {k: [round(n / args.steps, 1), round(ms / args.steps, 4)] for k, (n, ms) in st.items() if n}
    print(json.dumps({"only": "batch", "ms_per_run": graph_ms, "info": info, "eager_classes_launches_ms": per_run,
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--compute", default="TF32_RN", choices=["TF32X3", "F32", "BF16", "TF32", "MIXED", "TF32_MIXED", "TF32_RN"],
                    help="headline arithmetic: TF32_RN = TF32 Krylov blocks + a final pass on operands rounded to "
                         "nearest TF32 (default); MIXED = TF32 Krylov blocks + 3xTF32 final pass")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched (512-problem) leg")
    ap.add_argument("--no-completion", action="store_true", help="skip the matrix-completion leg")
    ap.add_argument("--no-sweep", action="store_true", help="skip the random low-rank size sweep")
    ap.add_argument("--no-legs", action="store_true", help="headline only (no peaks / mixed / sweeps / batched)")
    ap.add_argument("--only", choices=["sketch", "qsvd", "batch", "complete", "peaks"], default=None,
                    help="profiling driver: time only sketch passes, single QSVDs, batch runs or probes")
    ap.add_argument("--config", choices=["c2", "c3", "c4"], default="c4")
    ap.add_argument("--op", choices=["N", "H"], default="N")
    ap.add_argument("--ell", type=int, default=0)
    ap.add_argument("--m", type=int, default=0, help="profiling driver: rows of a uniform pure A (with --n)")
    ap.add_argument("--n", type=int, default=0, help="profiling driver: columns of a uniform pure A (with --m)")
    ap.add_argument("--passes", type=int, default=4)
    ap.add_argument("--noalloc", action="store_true",
                    help="profiling driver, --only sketch: time the allocation-free entry point instead")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.compute == "TF32_MIXED":
        args.compute = "MIXED"
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

    from paper_2507_13731_gb300 import build, qlr
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    golden = _golden()
    legs = ws == 1 and not args.no_legs
    peaks = peaks_leg(dev) if legs else None
    P = colour_problem()
    compute = getattr(qlr, "COMPUTE_" + args.compute)
    A_host = torch.from_numpy(np.ascontiguousarray(P.A[1:])).float().contiguous().pin_memory()
    Om_host = torch.from_numpy(np.ascontiguousarray(P.Omega.transpose(0, 2, 1))).float().contiguous().pin_memory()
    A = A_host.to(dev, non_blocking=True)
    om_store = Om_host.to(dev, non_blocking=True)
    om = om_store.transpose(1, 2)                                    # column-major n x l view
    U = qlr.empty_thin(HM, HK, device=dev)
    V = qlr.empty_thin(HN, HK, device=dev)
    S = torch.zeros(HK, dtype=torch.float64, device=dev)
    ctx = qlr.Context(local)
    ctx.reserve(qlr.workspace_size(HM, HN, HK, HB - HK, HV, qlr.ALG4, compute))

    def step():
        qlr.qsvd_lowrank(ctx, A, HK, HB - HK, HV, om, U, S, V, algo=qlr.ALG4, compute=compute, side=qlr.SIDE_X)

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
        step()
    t1e.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ctx.set_timing(False)
    elapsed_ms = t0e.elapsed_time(t1e)
    stats = ctx.stats()
    rc = ctx.sync()
    elapsed_ms = max_over_ranks(elapsed_ms, ws, dev)
    widths = [HB] * (HV - 1) + [HB * (HV // 2)]
    passes_per_step = len(widths)
    value = whole_job_rate(passes_per_step * args.steps, ws, elapsed_ms)
    a_bytes = A.numel() * A.element_size()
    tbs = ws * passes_per_step * args.steps * a_bytes / (elapsed_ms / 1e3) / 1e12
    gpu_launches = sum(n for n, _ in stats.values())
    S_gpu = S.cpu().numpy()

    # end to end through the C ABI with host buffers: H2D of A and Omega, D2H of U, S, V per step.
    # Two device input buffers: step i + 1's inputs are copied while step i computes (a stream of
    # QSVDs, each with its own host input); the first copy is exposed.  A's planes are copied on
    # streams of their own, so the copies run on several copy engines at once.
    U_h = torch.empty(4, HK, HM, dtype=torch.float32).pin_memory()
    V_h = torch.empty(4, HK, HN, dtype=torch.float32).pin_memory()
    S_h = torch.empty(HK, dtype=torch.float64).pin_memory()
    e2e_steps = max(2, args.steps)
    A_b = [A, torch.empty_like(A)]
    om_b = [om_store, torch.empty_like(om_store)]
    main = torch.cuda.current_stream(dev)
    cs = [torch.cuda.Stream(dev) for _ in range(A.shape[0])]
    ready = [[torch.cuda.Event() for _ in cs] for _ in range(2)]
    free = [torch.cuda.Event(), torch.cuda.Event()]

    def load(i):
        b = i % 2
        for c, st in enumerate(cs):
            if i >= 2:
                st.wait_event(free[b])             # step i - 2 has finished reading buffer b
            with torch.cuda.stream(st):
                A_b[b][c].copy_(A_host[c], non_blocking=True)
                if c == 0:
                    om_b[b].copy_(Om_host, non_blocking=True)
            ready[b][c].record(st)

    def e2e_run(nsteps):
        load(0)
        for i in range(nsteps):
            if i + 1 < nsteps:
                load(i + 1)
            b = i % 2
            for ev in ready[b]:
                main.wait_event(ev)
            qlr.qsvd_lowrank(ctx, A_b[b], HK, HB - HK, HV, om_b[b].transpose(1, 2), U, S, V, algo=qlr.ALG4,
                             compute=compute, side=qlr.SIDE_X)
            free[b].record(main)
            U_h.copy_(U.transpose(1, 2), non_blocking=True)
            V_h.copy_(V.transpose(1, 2), non_blocking=True)
            S_h.copy_(S, non_blocking=True)

    e2e_run(2)                                     # untimed: first use of the streams and buffers
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for st in cs:
        st.wait_event(e0)                          # the first copies start inside the timed region
    e2e_run(e2e_steps)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    # the inputs' copy alone (the same streams), for the line's information
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(main)
    for st in cs:
        st.wait_event(h0)
    load(1)
    for ev in ready[1]:
        main.wait_event(ev)
    h1.record(main)
    torch.cuda.synchronize()
    h2d_ms = h0.elapsed_time(h1)
    e2e_ms = max_over_ranks(e2e_ms, ws, dev)
    e2e_value = whole_job_rate(passes_per_step * e2e_steps, ws, e2e_ms)
    h2d = A_host.numel() * A_host.element_size() + Om_host.numel() * Om_host.element_size()
    d2h = U_h.numel() * 4 + V_h.numel() * 4 + S_h.numel() * 8

    line = None
    if rank == 0:
        total_ms = max(sum(t for _, t in stats.values()), 1e-9)
        roofs = []
        for kid, comp, ws_ in sketch_classes(args.compute, widths):
            nl, kms = stats[kid]
            if not nl:
                continue
            flops, nbytes = sketch_work(HM, HN, ws_ * args.steps, True, 4)
            r = sketch_roofline(flops, nbytes, kms, nl, comp, traffic_for(f"{kid}_{comp.lower()}_c4"))
            r.update({"class": kid, "compute": comp, "pass_widths": ws_, "class_share": round(kms / total_ms, 4)})
            roofs.append(r)
        roof = dict(max(roofs, key=lambda r: r["class_share"]))   # the sketch class with most time
        roof["dominant_class"] = max(stats, key=lambda k: stats[k][1])
        roof["sketch_classes"] = roofs
        errs = errors_vs_oracle(ctx, A, P, S_gpu, qlr.ALG4, HV, compute, golden.get("c4", {}).get("v6"))
        fp32_final = None
        if args.compute == "TF32_RN" and legs:
            # the same QSVD with the final pass in 3xTF32 (FP32-accurate for any singular vectors)
            def step_x3():
                qlr.qsvd_lowrank(ctx, A, HK, HB - HK, HV, om, U, S, V, algo=qlr.ALG4, compute=qlr.COMPUTE_TF32_MIXED,
                                 side=qlr.SIDE_X)
            for _ in range(2):
                step_x3()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record()
            for _ in range(5):
                step_x3()
            f1.record()
            torch.cuda.synchronize()
            fms = f0.elapsed_time(f1) / 5
            gs = golden.get("c4", {}).get("v6")
            fp32_final = {"compute": "MIXED (TF32 Krylov blocks, 3xTF32 final pass)", "ms_per_qsvd": round(fms, 3),
                          "sketch_passes_per_s": round(passes_per_step / (fms / 1e3), 3),
                          "sigma_rel_err": float(f"{sigma_rel_err(S.cpu().numpy(), gs['sigma']):.3e}") if gs else None,
                          "device_error": ctx.sync()}
        cpu = mixed = sweep2 = batched = completion = sweep = library = None
        if legs:
            for name, fn in (("library", lambda: library_leg(ctx, A)),
                             ("mixed", lambda: mixed_precision_leg(dev, golden)),
                             ("sweep2", lambda: pass_sweep_leg(dev, golden)),
                             ("batched", None if args.no_batched else lambda: batched_leg(dev)),
                             ("completion", None if args.no_completion else lambda: completion_leg(dev, golden)),
                             ("sweep", None if args.no_sweep else lambda: lowrank_sweep_leg(dev))):
                if fn is None:
                    continue
                try:
                    res = fn()
                except Exception as e:                 # reported, never fatal to the headline line
                    res = {"error": f"{type(e).__name__}: {e}"}
                if name == "library":
                    library = res
                elif name == "mixed":
                    mixed = res
                elif name == "sweep2":
                    sweep2 = res
                elif name == "batched":
                    batched = res
                elif name == "completion":
                    completion = res
                else:
                    sweep = res
        if ws == 1 and not args.no_cpu_baseline:
            val, secs, thr = cpu_oracle_sample(P)
            cpu = {"value": round(val, 5), "unit": "sketch passes/s", "cores": thr, "kind": "oracle",
                   "sample": f"one view of Algorithm 4 on the full matrix: Y = X Omega (60 columns) and the "
                             f"Householder QR of Y ({secs:.1f} s)"}
        dtypes = {"TF32X3": "f32 (3xTF32 tensor-core sketch, FP32 accumulation; FP64-class Gram and Cholesky)",
                  "MIXED": "f32/tf32 (TF32 sketches for the Krylov blocks, 3xTF32 for the final pass; FP64-class "
                           "Gram and Cholesky)",
                  "TF32_RN": "f32/tf32 (TF32 sketches for the Krylov blocks, operands rounded to nearest TF32 with "
                             "chunked FP32 sums for the final pass; FP64-class Gram and Cholesky)",
                  "F32": "f32 (SIMT)", "TF32": "tf32", "BF16": "bf16"}
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "sketch passes/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtypes[args.compute], "data": "synthetic",
            "config": {"workload": WORKLOAD, "compute": args.compute, "passes_per_step": passes_per_step,
                       "pass_widths": widths,
                       "l2": "inputs larger than L2 (A = %.0f MB > 129 MB L2)" % (a_bytes / 1e6),
                       "parallelism": f"replicas x{ws}"},
            "a_read_tbs": round(tbs, 4),
            "qsvd_ms": round(elapsed_ms / args.steps, 3),
            "error_vs_oracle": errs,
            "tolerance": {"sigma_rel": 1e-4},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_value, 3), "unit": "sketch passes/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps, "ms": round(e2e_ms, 3),
                    "h2d_ms_alone": round(h2d_ms, 3),
                    "overlap": "step i+1's H2D copies (one stream per plane of A) during step i (two device "
                               "input buffers); the first step's copy is exposed"},
            "gpu_launches": gpu_launches,
            "fp32_final_pass": fp32_final,
            "library_reference": library,
            "peaks": peaks,
            "mixed_precision": mixed,
            "pass_sweep": sweep2,
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
