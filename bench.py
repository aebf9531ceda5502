#!/usr/bin/env python
"""Throughput of batched Matcha rotational alignment on GB300.

Workload: 1024 (particle, template) pairs of 64^3 Gaussian-blob volumes
(48 blobs, sigma 2, SNR 0.1, +-60 degree missing wedge), 32 shells, SOFFT at
L0 = 8 with K = 2 and the top 16 candidates, Newton levels 8 -> 16 -> 24 -> 32
with 3 steps each.  A step is one pass of the whole path (shell sampling + SH
analysis of both volumes, contraction, SOFFT grid, top-P, Newton march, final
argmax) over the batch, inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl matcha|reference]

Prints one JSON line (rank 0).  Under torchrun each rank aligns its own 1024
particles (weak scaling, no data-path collective).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles aligned/sec at 64^3, final L=32 (ang. err ≤0.05° vs FP64 oracle)"
UNIT = "particles/s"
WORKLOAD = "batch64"
# FP32 ops per Wigner recurrence step, counted from the Newton kernel source
# (an FMA counts 2): derivative evaluation 20 (d, d', d'' recurrence) + 24
# (12 FMA accumulations); value-only evaluation 5 + 8.
# flops per (order pair, degree, candidate) step of the refinement's recurrences, counted
# from the source: a derivative step accumulates c d, c d', -l(l+1) c d (12 flops per
# complex pair of sums) and advances d and d' (11); a value-only step accumulates c d (8)
# and advances d (5)
FLOPS_FULL_STEP = 36
FLOPS_VALUE_STEP = 13
SMS, FP32_LANES = 152, 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="matcha", choices=["matcha", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "tf32", "bf16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    ap.add_argument("--no-pose6d", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-study", action="store_true")
    ap.add_argument("--no-oracle-gate", action="store_true",
                    help="skip the oracle run over the whole batch (accuracy against the oracle)")
    ap.add_argument("--batch", type=int, default=None, help="override particles per GPU")
    ap.add_argument("--stages", action="store_true",
                    help="time each entry point of the path once per stage on the batch (one "
                         "launch per stage, the SOFFT grid kept on chip) and exit: the "
                         "command the kernel profiles are captured with")
    ap.add_argument("--paper-batch", type=int, default=256, help="particles of the 200^3 leg")
    ap.add_argument("--pose6d-batch", type=int, default=1024, help="particles of the 6-D leg")
    return ap.parse_args()


from paper_2603_15285_gb300.shard import (aggregate_rate, barrier as rank_barrier, dist_env,
                                          max_over_ranks, shard_start)


def workload_config(w, B, ws):
    return {
        "workload": "%s: %d (particle, template) pairs of %d^3 float32 Gaussian-blob volumes per GPU "
                    "(%d blobs, sigma %.1f, SNR %.2f, wedge +-%d deg), %d shells, SOFFT L0=%d K=%d "
                    "top-%d, Newton L=%s x%d" % (w.name, B, w.N, w.n_blobs, w.sigma, w.snr,
                                                  int(w.wedge_deg), w.n_shells, w.L0, w.K, w.P,
                                                  "->".join(map(str, w.L_sched)), w.M_iter),
        "particles_per_gpu": B, "box": w.N, "shells": w.n_shells, "L_final": w.L_final,
        "L0": w.L0, "K": w.K, "P": w.P, "M_iter": w.M_iter,
        "parallelism": "dp%d (particles sharded, no collective)" % ws,
        "l2": l2_note(2 * B * w.N ** 3 * 4),
    }


def l2_note(nbytes):
    """Whether a step's inputs exceed the GB300's 129 MB L2 (no flush needed)."""
    if nbytes > 129e6:
        return "inputs %.1f GiB per step > 129 MB L2; no flush" % (nbytes / 2 ** 30)
    return "inputs %.0f MB per step, below the 129 MB L2" % (nbytes / 1e6)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def newton_traffic(B):
    """DRAM bytes per Newton launch from the committed ncu capture, scaled to
    B particles; None when the kernel source changed since the capture."""
    import hashlib
    try:
        meta = json.load(open(os.path.join(ROOT, "profiles", "k_newton_traffic.json")))
        src = open(os.path.join(ROOT, meta["source"]), "rb").read()
    except (OSError, ValueError, KeyError):
        return None
    if hashlib.sha256(src).hexdigest() != meta.get("sha256"):
        return None
    return meta["dram_bytes_per_launch_1024"] * B / 1024.0


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def oracle_near_ties(ref, rel=1e-6, distinct_deg=1.0):
    """Particles whose two best refined oracle candidates lie in different basins
    (rotations more than distinct_deg apart) with scores within rel of each
    other: for them the argmax may legitimately differ between paths."""
    import oracle
    ties = np.zeros(len(ref["score"]), dtype=bool)
    for b in range(len(ref["score"])):
        sc, eu = ref["cand_score"][b], ref["cand_euler"][b]
        k = int(ref["n_cand"][b])
        if k < 2:
            continue
        order = np.argsort(-sc[:k], kind="stable")
        Rb = oracle.euler_to_matrix(*eu[order[0]])
        for q in order[1:]:
            if math.degrees(oracle.rotation_angle(oracle.euler_to_matrix(*eu[q]), Rb)) > distinct_deg:
                ties[b] = sc[order[0]] - sc[q] < rel * abs(sc[order[0]])
                break
    return ties


def accuracy_vs_oracle(Rs, ref, R_true, ties):
    """Angular error of each path's refined rotations against the FP64 oracle
    (every particle; near-ties reported apart) and of the oracle against the
    planted rotation."""
    import oracle
    B = len(ref["score"])
    out = {"particles": B, "near_ties": int(ties.sum()),
           "near_tie_rule": "two best oracle candidates in different basins (> 1 deg apart) "
                            "with scores within 1e-6 relative"}
    keep = ~ties
    for name, R in Rs.items():
        e = np.degrees([oracle.rotation_angle(R[b], ref["R"][b]) for b in range(B)])
        out[name] = {"max_deg": float(e[keep].max()) if keep.any() else None,
                     "p90_deg": float(np.percentile(e[keep], 90)) if keep.any() else None,
                     "over_0.05deg": int((e[keep] > 0.05).sum()),
                     "max_deg_near_ties": float(e[ties].max()) if ties.any() else None}
    t = np.degrees([oracle.rotation_angle(ref["R"][b], R_true[b]) for b in range(B)])
    out["oracle_vs_planted_deg"] = {"median": float(np.median(t)), "p90": float(np.percentile(t, 90)),
                                    "max": float(t.max())}
    return out


def measure_fp32_peak(st, local, reps=5):
    """FP32 FMA throughput of this GPU, measured: independent FMA chains in
    every thread of 8 CTAs of 256 threads per SM (the probe in
    csrc/peak_probe.cu), timed with CUDA events on the launching stream, best of
    `reps` launches of about 25 ms; paired FP32x2 and scalar FMAs.  Returns
    TFLOP/s and the SM clock sampled during the probe."""
    import ctypes
    import torch
    from paper_2603_15285_gb300 import build as lib_build
    probe = ctypes.CDLL(lib_build.PROBE)
    probe.peak_fp32_launch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long,
                                       ctypes.c_void_p, ctypes.c_void_p]
    blocks, threads, iters = SMS * 8, 256, 200000
    buf = torch.empty(blocks * threads, dtype=torch.float32, device="cuda")
    flops = float(blocks) * threads * iters * 32
    out = {"probe": "csrc/peak_probe.cu: %d CTAs x %d threads, %d trips of 16 FMA lanes, best of %d"
                    % (blocks, threads, iters, reps)}
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.2)
    for name, variant in (("ffma2", 1), ("ffma", 0)):
        best = None
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            rc = probe.peak_fp32_launch(variant, blocks, threads, iters, buf.data_ptr(), st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            if rc != 0:
                raise RuntimeError("peak probe launch failed: %d" % rc)
            if r:
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
        out[name + "_tflops"] = flops / (best * 1e-3) / 1e12
    out["clocks"] = sampler.stop()
    return out


def wigner_term_units(w, B, newton_ms, peak):
    """Newton's work in Wigner terms, 3 P sum_j T(L_j) per particle with
    T(L) = (L+1)(2L+1)(2L+3)/3, at 30 flops per term (the per-unit figure of
    the path's roofline table), against the ALU peak."""
    T = lambda L: (L + 1) * (2 * L + 1) * (2 * L + 3) // 3
    terms = 3 * w.P * sum(T(L) for L in w.L_sched)
    ach = 30.0 * terms * B / (newton_ms * 1e-3) / 1e12
    return {"wigner_terms_per_particle": terms, "flops_per_term": 30, "achieved": ach,
            "unit": "TFLOP/s", "frac": ach / peak}


def kernel_roofline(w, B, prec, stage_ms, alu_peak, m):
    """Achieved fraction of each step's bound, from the event-timed stages and
    the algorithmic work per particle (volume bytes for the analysis, with its
    dense DFT and Legendre flops beside them, 8 S T(L) flops for the
    contraction, grid points for the SOFFT search)."""
    pk = measured_peaks()
    hbm = pk["hbm_gbs"]
    L, S, N = w.L_sched[-1], w.n_shells, w.N
    T = (L + 1) * (2 * L + 1) * (2 * L + 3) // 3
    vol_bytes = 2 * 4 * N ** 3 * B  # particle + template volumes, read once
    out = {"analysis": {"kernel": "k_analyze2 (x2)", "bound": "hbm", "unit": "GB/s", "peak": hbm,
                        "achieved": vol_bytes / (stage_ms["analyze"] * 1e-3) / 1e9}}
    out["analysis"]["frac"] = out["analysis"]["achieved"] / hbm
    # the same launches in flops: per volume and shell, the phi DFT of n_theta
    # rings of n_phi real samples to L+1 orders and the Legendre sums of n_lm
    # coefficients over n_theta nodes, 4 flops per complex multiply-add
    nt, nphi, nlm_a = L + 1, 2 * L + 2, (L + 1) * (L + 2) // 2
    an_flops = 2.0 * S * (4 * nt * nphi * (L + 1) + 4 * nlm_a * nt) * B
    out["analysis"]["flops_per_particle"] = an_flops / B
    out["analysis"]["alu_frac"] = an_flops / (stage_ms["analyze"] * 1e-3) / 1e12 / alu_peak
    flops = 8.0 * S * T * B
    if prec in (m.TF32, m.BF16):
        tpk = pk["bf16_tflops"] * (1.0 if prec == m.BF16 else 1.1 / 2.25)
        src = "measured bf16 burst" + ("" if prec == m.BF16 else " x 1.1/2.25 (nominal TF32/BF16 ratio)")
        out["contraction"] = {"kernel": "k_correlate_tc", "bound": "tensor", "unit": "TFLOP/s",
                              "peak": tpk, "peak_source": src}
    else:
        out["contraction"] = {"kernel": "k_correlate_deg", "bound": "alu", "unit": "TFLOP/s",
                              "peak": alu_peak, "peak_source": "the roofline's ALU peak"}
    c = out["contraction"]
    c["achieved"] = flops / (stage_ms["correlate"] * 1e-3) / 1e12
    c["frac"] = c["achieved"] / c["peak"]
    # bytes the contraction must move: f, h (complex S x n_lm) and c (grouped entries)
    rb = 8 if prec == m.FP64 else 4
    nlm = (L + 1) * (L + 2) // 2
    ge = sum((mm + 1) * (L - mm + 1) for mm in range(L + 1))
    c["hbm_frac"] = (2 * S * nlm * 2 * rb + 8 * ge * rb) * B / (stage_ms["correlate"] * 1e-3) / 1e9 / hbm
    n = 2 * w.K * (w.L0 + 1)
    # SOFFT work per particle: the beta transform, 4 flops per (beta_k, l, m, n)
    # term (complex coefficient times real d), plus one real-output 2-D FFT of
    # n x n points per beta slice at 2.5 n^2 log2(n^2) flops (half the complex
    # 5 N log2 N count); the kernel's direct separable DFT executes more
    T0 = (w.L0 + 1) * (2 * w.L0 + 1) * (2 * w.L0 + 3) // 3
    soft_flops = (4.0 * n * T0 + 2.5 * n ** 3 * math.log2(n * n)) * B
    sp = alu_peak
    tiled = prec != m.FP64 and w.L0 == 8 and n == 36  # the register-tiled kernel's plans
    out["soft"] = {"kernel": "k_soft_tile" if tiled else "k_soft_chunk", "bound": "alu",
                   "unit": "TFLOP/s", "peak": sp,
                   "flops_per_particle": soft_flops / B,
                   "achieved": soft_flops / (stage_ms["soft"] * 1e-3) / 1e12,
                   "grid_points_per_s": n ** 3 * B / (stage_ms["soft"] * 1e-3)}
    out["soft"]["frac"] = out["soft"]["achieved"] / sp
    out["peaks_file"] = pk.get("source", "MEASURED_PEAKS.json")
    return out


def time_backward(st, reps=5):
    """Template gradient of the refined scores on the shared-template 64^3
    workload (512 particles, L 8 -> 32): forward (a1..a7 from the template's
    and particles' analyses) and matcha_template_grad timed apart, FP32 and
    FP64 plans; the gradient itself is checked against the oracle's adjoint
    and central differences in the tests."""
    import torch
    import paper_2603_15285_gb300 as m
    import synth
    wg = synth.WORKLOADS["grad64"]
    d = synth.make_batch(wg, device="cuda")
    parts, temp = d["particles"], d["templates"]
    out = {"workload": "grad64: %d particles, one shared %d^3 template, S=%d, L %s, P=%d"
                       % (wg.B, wg.N, wg.n_shells, "->".join(map(str, wg.L_sched)), wg.P)}
    for name, prec in (("fp32", m.FP32), ("fp64", m.FP64)):
        plan = m.plan_for_workload(wg, precision=prec)
        f = m.matcha_analyze(plan, parts)
        h = m.matcha_analyze(plan, temp)
        fw = m.align_from_coefs(plan, f, h, 0)
        m.matcha_template_grad(plan, f, fw["c"], fw["euler"])
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(st)
        for _ in range(reps):
            fw = m.align_from_coefs(plan, f, h, 0)
        e[1].record(st)
        for _ in range(reps):
            g = m.matcha_template_grad(plan, f, fw["c"], fw["euler"])
        e[2].record(st)
        torch.cuda.synchronize()
        fms, bms = e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps
        out[name] = {"forward_ms": fms, "backward_ms": bms,
                     "backward_particles_per_s": wg.B / (bms * 1e-3),
                     "singular_hessians": int((g["flags"] != 0).sum().item())}
        plan.close()
    return out


def time_mixed(st, prec, reps=5):
    """The mixed-size batch (2048 x 48^3 / L 24, 1024 x 64^3 / L 32, 1024 x
    96^3 / L 48; per-particle SNR and candidate counts): autotuned plans, all
    groups captured in one CUDA graph (concurrent streams, costliest first)
    and replayed."""
    import torch
    import paper_2603_15285_gb300 as m
    import synth
    from paper_2603_15285_gb300 import mixed
    groups, total = [], 0
    for name in ("var48", "var64", "var96"):
        w = synth.WORKLOADS[name]
        d = synth.make_batch(w, device="cuda")
        groups.append(dict(plan=m.plan_for_workload(w, precision=prec),
                           particles=d["particles"].contiguous(),
                           templates=d["templates"].contiguous(),
                           P_per=torch.from_numpy(d["P_per"]).to("cuda")))
        total += w.B
    mb = mixed.MixedBatch(groups, autotune=True).capture()
    for _ in range(2):
        mb.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        mb.replay()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"workload": "mixed: 2048 x 48^3 (S 24, L 8..24) + 1024 x 64^3 (S 32, L 8..32) + "
                        "1024 x 96^3 (S 48, L 8..48), P_b ~ U{8..32}, SNR ~ U[0.05, 0.3]",
            "particles": total, "ms_per_step": ms, "value": total / (ms * 1e-3),
            "unit": "particles/s", "timed": "one CUDA graph of all groups, replayed",
            "autotune": [{"shells_per_analysis_cta": t["analyze_shells"],
                          "tc_ctas_per_sm": t["tc_ctas_per_sm"],
                          "soft_kernel": t.get("soft_kernel", 0),
                          "newton_sched": t.get("newton_sched", 0),
                          "newton_ms": t.get("newton_ms")} for t in mb.tune]}


def time_paper_scale(st, reps=3, n=256):
    """The paper's own regime (200^3 boxes, 40 shells, SOFFT at L0 = 30 with
    K = 2, P = 10, one Newton step per band, L 30 -> 40, 0 dB): FP32 and FP64
    plans, eager matcha_align, errors against FP64 and the planted rotation."""
    import numpy as np
    import torch
    import oracle
    import paper_2603_15285_gb300 as m
    import synth
    w = synth.WORKLOADS["paper200"]
    d = synth.make_batch(w, B=n, device="cuda")
    parts, temps = d["particles"].contiguous(), d["templates"].contiguous()
    B = parts.shape[0]
    out = {"workload": "paper200: %d particles of 200^3, 40 shells, L0=30 K=2 (124^3 grid), P=10, "
                       "L 30->40, one Newton step per band, SNR 1 (0 dB), +-60 deg wedge" % B}
    Rs = {}
    for name, prec in (("fp32", m.FP32), ("fp64", m.FP64)):
        plan = m.plan_for_workload(w, precision=prec)
        ws = m.alloc_workspace(plan, B)
        o = m.matcha_align(plan, parts, temps, ws=ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            m.matcha_align(plan, parts, temps, ws=ws, out=o)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms_per_step": ms, "value": B / (ms * 1e-3), "unit": "particles/s"}
        Rs[name] = o["R"].cpu().numpy()
        del ws
        plan.close()
    e = np.degrees([oracle.rotation_angle(Rs["fp32"][b], Rs["fp64"][b]) for b in range(B)])
    t = np.degrees([oracle.rotation_angle(Rs["fp64"][b], d["R_true"][b]) for b in range(B)])
    out["fp32_vs_fp64_deg"] = {"max": float(e.max()), "p90": float(np.percentile(e, 90))}
    out["fp64_vs_planted_deg"] = {"median": float(np.median(t)), "p90": float(np.percentile(t, 90)),
                                  "max": float(t.max())}
    return out


def time_pose6d(st, reps=3, n=None):
    """6-D pose (rotation and translation) on the 1024-particle 64^3 batch with
    planted shifts up to 3 voxels: three rotation-translation alternations
    (matcha_align6d: per round the rotation search, the rotated template, the
    box FFT correlation, the integer window +-5 and the 1/10-voxel grid),
    FP32 plan, eager calls; errors against the planted pose."""
    import torch
    import oracle
    import paper_2603_15285_gb300 as m
    import synth
    w = synth.WORKLOADS["shift64"]
    d = synth.make_batch(w, B=n, device="cuda")
    parts, temps = d["particles"].contiguous(), d["templates"].contiguous()
    B = parts.shape[0]
    plan = m.plan_for_workload(w, precision=m.FP32)
    ws = m.alloc_workspace6d(plan, B, 1, w.max_shift, 10)
    o = m.matcha_align6d(plan, parts, temps, w.rounds, w.max_shift, 10, ws=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        m.matcha_align6d(plan, parts, temps, w.rounds, w.max_shift, 10, ws=ws, out=o)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # the translation search alone (one round's share), on the final rotations
    rot = m.matcha_transform_volumes(temps, o["R"], precision=m.FP32)
    sw = m.matcha_shift_search(plan, parts, rot, w.max_shift, 10, R=o["R"])
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        m.matcha_shift_search(plan, parts, rot, w.max_shift, 10, R=o["R"])
    e1.record(st)
    torch.cuda.synchronize()
    ms_shift = e0.elapsed_time(e1) / reps
    R = o["R"].cpu().numpy()
    tau = o["tau"].cpu().numpy()
    ang = np.degrees([oracle.rotation_angle(R[b], d["R_true"][b]) for b in range(B)])
    sh = np.linalg.norm(tau - d["tau_true"], axis=1)
    del ws
    plan.close()
    return {"workload": "shift64: %d pairs of 64^3, planted shifts |tau*| <= 3 vox, %d rounds, "
                        "window +-%d, 1/10-voxel grid, FP32" % (B, w.rounds, w.max_shift),
            "ms_per_step": ms, "value": B / (ms * 1e-3), "unit": "particles/s",
            "shift_search_ms": ms_shift,
            "vs_planted": {"angle_deg_median": float(np.median(ang)),
                           "angle_deg_p90": float(np.percentile(ang, 90)),
                           "shift_vox_median": float(np.median(sh)),
                           "shift_vox_p90": float(np.percentile(sh, 90))}}


def time_precision(st, reps=2, sample=8):
    """The precision workload (2048 pairs of 64^3, S = 32, final L = 48):
    matcha_align timed in FP64, FP32, TF32 and BF16 plans (eager), and for a
    sample of particles the error of every path against the FP64 oracle:
    the refined rotation against the oracle's whole path, and C_L, its
    gradient and Hessian (matcha_objective on the path's own coefficients)
    against the oracle's objective at the path's refined rotation."""
    import torch
    import oracle
    import paper_2603_15285_gb300 as m
    import synth
    w = synth.WORKLOADS["deep64"]
    d = synth.make_batch(w, device="cuda")
    parts, temps = d["particles"].contiguous(), d["templates"].contiguous()
    B = parts.shape[0]
    L, S, R = w.L_sched[-1], w.n_shells, w.r_max
    ps, ts = parts[:sample].cpu().numpy(), temps[:sample].cpu().numpy()
    ref = oracle.align_batch(ps, ts, S=S, r_max=R, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter,
                             L_sched=w.L_sched)
    cor = [oracle.correlate(oracle.analyze_volume(ps[b], S, R, L), oracle.analyze_volume(ts[b], S, R, L),
                            S, R, L) for b in range(sample)]
    out = {"workload": "deep64: %d pairs of 64^3, S=%d, L %s, P=%d; errors on the first %d particles"
                       % (B, S, "->".join(map(str, w.L_sched)), w.P, sample)}
    for name, prec in (("fp64", m.FP64), ("fp32", m.FP32), ("tf32", m.TF32), ("bf16", m.BF16)):
        plan = m.plan_for_workload(w, precision=prec)
        ws = m.alloc_workspace(plan, B)
        o = m.matcha_align(plan, parts, temps, ws=ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = 1 if prec == m.FP64 else reps
        e0.record(st)
        for _ in range(k):
            m.matcha_align(plan, parts, temps, ws=ws, out=o)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        del ws
        eu = o["euler"][:sample].contiguous()
        f = m.matcha_analyze(plan, parts[:sample].contiguous())
        h = m.matcha_analyze(plan, temps[:sample].contiguous())
        c = m.matcha_correlate_coeffs(plan, f, h, 1)
        ob = m.matcha_objective(plan, c, eu[:, None, :].contiguous()).cpu().numpy()[:, 0]
        Rg = o["R"][:sample].cpu().numpy()
        ang, eC, eg, eH = [], [], [], []
        for b in range(sample):
            C, g, H, _ = oracle.objective(cor[b], L, *eu[b].cpu().numpy(), derivs=True)
            eC.append(abs(ob[b, 0] - C) / abs(C))
            eg.append(np.abs(ob[b, 1:4] - g).max() / abs(C))
            Hv = np.array([H[0, 0], H[0, 1], H[0, 2], H[1, 1], H[1, 2], H[2, 2]])
            eH.append(np.abs(ob[b, 4:] - Hv).max() / np.abs(Hv).max())
            ang.append(math.degrees(oracle.rotation_angle(Rg[b], ref["R"][b])))
        out[name] = {"ms_per_step": ms, "value": B / (ms * 1e-3), "unit": "particles/s",
                     "angle_deg_max_vs_oracle": max(ang), "C_rel_max": max(eC),
                     "grad_max_over_C": max(eg), "hessian_rel_max": max(eH)}
        plan.close()
    return out


def time_refine_study(st, n=128):
    """Section 5.1's comparisons on the 64^3 batch (first n particles, FP32):
    refinement by Newton steps against gradient steps at several step counts
    per level, and the dense SOFFT baseline (the best grid point, no
    refinement) at increasing oversampling K; angular error against the
    FP64 path's Newton result and against the planted rotation, and time."""
    import dataclasses
    import torch
    import oracle
    import paper_2603_15285_gb300 as m
    import synth
    w = synth.WORKLOADS[WORKLOAD]
    d = synth.make_batch(w, B=n, device="cuda")
    parts, temps = d["particles"].contiguous(), d["templates"].contiguous()
    p64 = m.plan_for_workload(w, precision=m.FP64)
    Rref = m.matcha_align(p64, parts, temps)["R"].cpu().numpy()
    p64.close()

    def timed(fn, k=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(k):
            r = fn()
        e1.record(st)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / k

    def errs(R):
        a = np.degrees([oracle.rotation_angle(R[b], Rref[b]) for b in range(n)])
        t = np.degrees([oracle.rotation_angle(R[b], d["R_true"][b]) for b in range(n)])
        return {"p90_deg_vs_fp64_newton": float(np.percentile(a, 90)), "max_deg_vs_fp64_newton": float(a.max()),
                "p90_deg_vs_planted": float(np.percentile(t, 90))}
    out = {"workload": "first %d particles of batch64, FP32" % n, "newton": {}, "gradient": {}, "dense_soft": {}}
    for refine, key, steps in ((0, "newton", (1, 2, 3, 5)), (1, "gradient", (1, 3, 10, 30))):
        for M in steps:
            plan = m.plan_for_workload(dataclasses.replace(w, M_iter=M), precision=m.FP32, refine=refine)
            ws = m.alloc_workspace(plan, n)
            o, ms = timed(lambda: m.matcha_align(plan, parts, temps, ws=ws))
            out[key]["M=%d" % M] = dict(errs(o["R"].cpu().numpy()), ms=ms)
            del ws
            plan.close()
    for K in (2, 4, 8, 16):
        wk = dataclasses.replace(w, K=K, P=1)
        plan = m.plan_for_workload(wk, precision=m.FP32)
        f = m.matcha_analyze(plan, parts)
        h = m.matcha_analyze(plan, temps)
        c = m.matcha_correlate_coeffs(plan, f, h, 1)
        grid = torch.empty((n,) + (plan.info.soft_n,) * 3, dtype=torch.float32, device="cuda")
        s, ms = timed(lambda: m.matcha_soft_search(plan, c, grid=grid))
        eu = s["euler"][:, 0].cpu().numpy()
        R = np.stack([oracle.euler_to_matrix(*eu[b]) for b in range(n)])
        out["dense_soft"]["K=%d" % K] = dict(errs(R), ms=ms, points_per_angle=plan.info.soft_n)
        del grid
        plan.close()
    return out


def host_cpu():
    """Model name of the host CPU from /proc/cpuinfo (Arm hosts give implementer
    and part codes instead of a name), else the platform's processor string."""
    import platform
    name, impl, part = "", "", ""
    try:
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            k, v = k.strip(), v.strip()
            if k == "model name" and not name:
                name = v
            elif k == "CPU implementer" and not impl:
                impl = v
            elif k == "CPU part" and not part:
                part = v
    except OSError:
        pass
    if name:
        return name
    if impl or part:
        arm = {"0xd0c": "Neoverse N1", "0xd40": "Neoverse V1", "0xd49": "Neoverse N2",
               "0xd4f": "Neoverse V2"}
        core = arm.get(part, "") if impl == "0x41" else ""
        return "%s (implementer %s, part %s%s)" % (platform.machine(), impl or "?", part or "?",
                                                   ": " + core if core else "")
    return platform.processor() or platform.machine()


def oracle_per_core(oracle, pc, tc, kw, n=3):
    """The oracle on one host thread, on the first n particles: the per-core rate."""
    t0 = time.perf_counter()
    oracle.align_batch(pc[:n], tc[:n] if tc.shape[0] == pc.shape[0] else tc, n_threads=1, **kw)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": 1,
            "sample": "first %d particles of the batch, one thread, %.1f s" % (n, dt)}


def run_reference(args):
    """The oracle (FP64 C, all host cores) on a bounded sample of the workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import synth
    import oracle
    w = synth.WORKLOADS[WORKLOAD]
    cores = oracle.max_threads()
    n = max(1, cores)
    d = synth.make_batch(w, B=n)
    parts, temps = d["particles"].numpy(), d["templates"].numpy()
    kw = dict(S=w.n_shells, r_max=w.r_max, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter, L_sched=w.L_sched)
    for _ in range(args.warmup):
        oracle.align_batch(parts[:1], temps[:1], **kw)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.align_batch(parts, temps, **kw)
    dt = (time.perf_counter() - t0) / args.steps
    v = n / dt
    sample = ("each step aligns a bounded sample of the %d-particle %s batch: its first %d "
              "particles, one per host thread, FP64 C oracle; the rate is particles per second"
              % (w.B, WORKLOAD, n))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w, w.B, 1),
        "timed_sample_per_step": n,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu": host_cpu()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_stages(args):
    """One launch per stage of the path through the C ABI on the batch (after
    `--warmup` untimed passes), each timed with CUDA events: analysis of the
    particles and templates, contraction, SOFFT search (allocation-free entry,
    grid on chip), Newton march from the search's candidates, final selection."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2603_15285_gb300 as m
    import synth
    w = synth.WORKLOADS[WORKLOAD]
    B = args.batch or w.B
    prec = {"fp32": m.FP32, "fp64": m.FP64, "tf32": m.TF32, "bf16": m.BF16}[args.precision]
    d = synth.make_batch(w, B=B, device="cuda")
    parts, temps = d["particles"].contiguous(), d["templates"].contiguous()
    plan = m.plan_for_workload(w, precision=prec)
    rt = plan.real_dtype
    f = torch.empty((B, w.n_shells, plan.info.n_lm, 2), dtype=rt, device="cuda")
    h = torch.empty_like(f)
    c = torch.empty((B, plan.info.corr_entries, 2, 2), dtype=rt, device="cuda")
    L, st, H = m.lib(), torch.cuda.current_stream(), plan.handle
    sp = st.cuda_stream
    idx = torch.empty((B, w.P), dtype=torch.int32, device="cuda")
    eu = torch.empty((B, w.P, 3), dtype=torch.float64, device="cuda")
    sc = torch.empty((B, w.P), dtype=torch.float64, device="cuda")
    fl = torch.empty((B, w.P), dtype=torch.int32, device="cuda")
    nc = torch.empty((B,), dtype=torch.int32, device="cuda")
    out = [torch.empty((B, k), dtype=t, device="cuda") for k, t in
           ((3, torch.float64), (9, torch.float64), (1, torch.float64), (1, torch.int32),
            (1, torch.int32))]
    e0, s0 = torch.empty_like(eu), torch.empty_like(sc)
    stages = {
        "analyze": lambda: (m._check(L.matcha_analyze(H, parts.data_ptr(), B, f.data_ptr(), sp), "a"),
                            m._check(L.matcha_analyze(H, temps.data_ptr(), B, h.data_ptr(), sp), "a")),
        "correlate": lambda: m._check(L.matcha_correlate_coeffs(H, f.data_ptr(), h.data_ptr(), B, 1,
                                                                c.data_ptr(), sp), "c"),
        "soft": lambda: (m._check(L.matcha_soft_search_noalloc(
            H, c.data_ptr(), B, None, idx.data_ptr(), eu.data_ptr(), sc.data_ptr(),
            nc.data_ptr(), sp), "s"), e0.copy_(eu), s0.copy_(sc)),
        "newton": lambda: m._check(L.matcha_newton_march(H, c.data_ptr(), B, nc.data_ptr(),
                                                         eu.data_ptr(), sc.data_ptr(),
                                                         fl.data_ptr(), None, sp), "n"),
        "select": lambda: m._check(L.matcha_final_select(
            H, B, None, nc.data_ptr(), eu.data_ptr(), sc.data_ptr(), fl.data_ptr(),
            *[o.data_ptr() for o in out], sp), "f"),
    }
    res = {}
    for name, fn in stages.items():
        for _ in range(args.warmup):
            if name == "newton":
                eu.copy_(e0); sc.copy_(s0)
            fn()
        if name == "newton":
            eu.copy_(e0); sc.copy_(s0)
        a = torch.cuda.Event(enable_timing=True); z = torch.cuda.Event(enable_timing=True)
        a.record(st); fn(); z.record(st)
        torch.cuda.synchronize()
        res[name] = a.elapsed_time(z)
    print(json.dumps({"stages_ms": res, "particles": B, "workload": WORKLOAD,
                      "precision": args.precision}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.stages:
        run_stages(args)
        return
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2603_15285_gb300 as m
    import synth
    w = synth.WORKLOADS[WORKLOAD]
    B = args.batch or w.B
    d = synth.make_batch(w, B=B, start=shard_start(rank, B), device="cuda")
    parts, temps = d["particles"].contiguous(), d["templates"].contiguous()
    PRECS = {"fp32": m.FP32, "fp64": m.FP64, "tf32": m.TF32, "bf16": m.BF16}
    prec = PRECS[args.precision]
    is32 = prec != m.FP64
    plan = m.plan_for_workload(w, precision=prec)
    n = plan.info.soft_n
    rt = plan.real_dtype
    f = torch.empty((B, w.n_shells, plan.info.n_lm, 2), dtype=rt, device="cuda")
    h = torch.empty_like(f)
    c = torch.empty((B, plan.info.corr_entries, 2, 2), dtype=rt, device="cuda")
    grid = torch.empty((B, n, n, n), dtype=rt, device="cuda")
    work = torch.zeros((B, 2), dtype=torch.int64, device="cuda")
    L = m.lib()
    st = torch.cuda.current_stream()
    sp = st.cuda_stream
    idx = torch.empty((B, w.P), dtype=torch.int32, device="cuda")
    ceu = torch.empty((B, w.P, 3), dtype=torch.float64, device="cuda")
    csc = torch.empty((B, w.P), dtype=torch.float64, device="cuda")
    cfl = torch.empty((B, w.P), dtype=torch.int32, device="cuda")
    ncd = torch.empty((B,), dtype=torch.int32, device="cuda")
    out = dict(euler=torch.empty((B, 3), dtype=torch.float64, device="cuda"),
               R=torch.empty((B, 3, 3), dtype=torch.float64, device="cuda"),
               score=torch.empty((B,), dtype=torch.float64, device="cuda"),
               best_p=torch.empty((B,), dtype=torch.int32, device="cuda"),
               flags=torch.empty((B,), dtype=torch.int32, device="cuda"))
    H = plan.handle
    stages = ["analyze", "correlate", "soft", "newton", "select"]
    # Kernels of one matcha_align step: per part of the batch k_analyze2 x2
    # (particles, templates), the contraction, k_soft_tile (grid and top-P
    # fused), k_newton, k_final_select; from 256 particles on the batch runs as
    # min(4, B / 128) concurrent parts (a shared template is analysed once).
    n_parts = 1 if B < 256 else min(4, B // 128)  # (batch64's SOFFT is fused)
    shared = temps.shape[0] != B
    KERNELS_PER_STEP = n_parts * (5 if shared else 6) + (1 if shared else 0)

    def step(ev=None):
        def mark(i):
            if ev is not None:
                ev[i].record(st)
        mark(0)
        m._check(L.matcha_analyze(H, parts.data_ptr(), B, f.data_ptr(), sp), "analyze")
        m._check(L.matcha_analyze(H, temps.data_ptr(), temps.shape[0], h.data_ptr(), sp), "analyze")
        mark(1)
        m._check(L.matcha_correlate_coeffs(H, f.data_ptr(), h.data_ptr(), B,
                                           1 if temps.shape[0] == B else 0, c.data_ptr(), sp), "corr")
        mark(2)
        m._check(L.matcha_soft_search(H, c.data_ptr(), B, None, grid.data_ptr(), idx.data_ptr(),
                                      ceu.data_ptr(), csc.data_ptr(), ncd.data_ptr(), sp), "soft")
        mark(3)
        m._check(L.matcha_newton_march(H, c.data_ptr(), B, ncd.data_ptr(), ceu.data_ptr(),
                                       csc.data_ptr(), cfl.data_ptr(), work.data_ptr(), sp), "newton")
        mark(4)
        m._check(L.matcha_final_select(H, B, None, ncd.data_ptr(), ceu.data_ptr(), csc.data_ptr(),
                                       cfl.data_ptr(), out["euler"].data_ptr(), out["R"].data_ptr(),
                                       out["score"].data_ptr(), out["best_p"].data_ptr(),
                                       out["flags"].data_ptr(), sp), "select")
        mark(5)

    def barrier():
        rank_barrier(ws)

    # The timed step is the user-facing call, matcha_align (a1..a7), replayed
    # from a CUDA graph (it is stream-ordered and allocates nothing); a second,
    # stage-wise pass through the individual entry points gives the per-stage
    # times and the Newton work counters.
    ws_a = m.alloc_workspace(plan, B)
    out_a = {k: torch.empty_like(v) for k, v in out.items()}

    def align_eager():
        m.matcha_align(plan, parts, temps, ws=ws_a, out=out_a)

    for _ in range(max(3, args.warmup)):
        align_eager()
    torch.cuda.synchronize()
    timed_how = "matcha_align (a1..a7) replayed from a CUDA graph"
    try:
        cs = torch.cuda.Stream()
        cs.wait_stream(st)
        with torch.cuda.stream(cs):
            align_eager()
        st.wait_stream(cs)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            align_eager()
        torch.cuda.synchronize()
        run_step = graph.replay
    except Exception as exc:  # capture unsupported here: time the eager calls
        run_step = align_eager
        timed_how = "matcha_align (a1..a7), eager (graph capture failed: %s)" % exc
    for _ in range(max(3, args.warmup)):
        run_step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(st)
    for k in range(args.steps):
        run_step()
    t_end.record(st)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(t_start.elapsed_time(t_end) / args.steps, ws, device="cuda")
    # stage-wise pass (not part of the timed value)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    for k in range(args.steps):
        step(evs[k])
    torch.cuda.synchronize()
    stage_ms = {s: statistics.mean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps))
                for i, s in enumerate(stages)}
    wk = work.sum(0).cpu().numpy()
    newton_flops = FLOPS_FULL_STEP * float(wk[0]) + FLOPS_VALUE_STEP * float(wk[1])
    clk = clocks.get("sm_max_mhz") or 2070.0
    fp32_derived = SMS * FP32_LANES * 2 * clk * 1e6 / 1e12  # TFLOP/s
    fp64_peak = SMS * 2 * 2 * clk * 1e6 / 1e12
    fp32_meas = measure_fp32_peak(st, local)
    fp32_peak = max(fp32_meas["ffma2_tflops"], fp32_meas["ffma_tflops"])
    achieved = newton_flops / (stage_ms["newton"] * 1e-3) / 1e12
    peak = fp32_peak if is32 else fp64_peak
    value = aggregate_rate(ws, B, ms * 1e-3)
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if is32 else "f64",
        "contraction": {m.FP32: "FP32 CUDA cores", m.FP64: "FP64 CUDA cores",
                        m.TF32: "tcgen05 TF32 operands, FP32 accumulation",
                        m.BF16: "tcgen05 BF16 operands, FP32 accumulation"}[prec],
        "data": "synthetic (seeded Gaussian-blob volumes; no dataset)",
        "config": workload_config(w, B, ws),
        "timed": timed_how,
        "stage_ms": stage_ms,
        "roofline": {"kernel": "k_newton", "bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": newton_traffic(B) if is32 else None,
                     "peak_source": ("measured FP32 FMA probe (of measured; derived %.1f = %d SMs x "
                                     "%d lanes x 2 x %.0f MHz)" % (fp32_derived, SMS, FP32_LANES, clk))
                                    if is32 else
                                    "%d SMs x 2 FP64 lanes x 2 x %.0f MHz (derived)" % (SMS, clk),
                     "flops_per_launch": newton_flops,
                     # the same launch in the path's algorithmic unit: 3 P sum_j T(L_j)
                     # Wigner terms per particle (three evaluations per level) at 30 flops
                     # per term, against the same peak
                     "wigner_term_units": wigner_term_units(w, B, stage_ms["newton"], peak)},
        "fp32_peak_probe": fp32_meas,
        "clocks": clocks,
        "gpu_launches": KERNELS_PER_STEP * args.steps,
    }
    res["kernel_roofline"] = kernel_roofline(w, B, prec, stage_ms, peak, m)
    Rs = {args.precision: out["R"].cpu().numpy()}  # refined rotations of each path
    # accuracy of the timed path against the FP64 GPU path (oracle-checked in the tests)
    if rank == 0 and not args.no_fp64 and is32:
        plan64 = m.plan_for_workload(w, precision=m.FP64)
        ws64 = m.alloc_workspace(plan64, B)
        o64 = m.matcha_align(plan64, parts, temps, ws=ws64)
        torch.cuda.synchronize()
        k64 = max(2, args.steps // 25)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(k64):
            m.matcha_align(plan64, parts, temps, ws=ws64, out=o64)
        e1.record(st)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / k64
        import oracle
        R32, R64 = out["R"].cpu().numpy(), o64["R"].cpu().numpy()
        Rs["fp64"] = R64
        errs = np.degrees([oracle.rotation_angle(R32[b], R64[b]) for b in range(B)])
        res["fp64_path"] = {"value": B / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                            "steps": k64}
        res["accuracy_vs_fp64_gpu"] = {"max_deg": float(errs.max()),
                                       "p90_deg": float(np.percentile(errs, 90))}
        del ws64
        # the other 32-bit plans (contraction on CUDA cores or tensor cores), eager timing
        others = {}
        for name, pr in (("fp32", m.FP32), ("tf32", m.TF32), ("bf16", m.BF16)):
            if pr == prec:
                continue
            po = m.plan_for_workload(w, precision=pr)
            wso = m.alloc_workspace(po, B)
            oo = m.matcha_align(po, parts, temps, ws=wso)
            torch.cuda.synchronize()
            e0.record(st)
            for _ in range(k64 * 5):
                m.matcha_align(po, parts, temps, ws=wso, out=oo)
            e1.record(st)
            torch.cuda.synchronize()
            mso = e0.elapsed_time(e1) / (k64 * 5)
            Ro = oo["R"].cpu().numpy()
            Rs[name] = Ro
            eo = np.degrees([oracle.rotation_angle(Ro[b], R64[b]) for b in range(B)])
            others[name] = {"value": B / (mso * 1e-3), "unit": UNIT, "ms_per_step": mso,
                            "timed": "matcha_align, eager", "max_err_deg_vs_fp64_gpu": float(eo.max()),
                            "p90_err_deg_vs_fp64_gpu": float(np.percentile(eo, 90))}
            del wso
            po.close()
        res["other_32bit_paths"] = others
    if not args.no_e2e:
        hp = torch.empty_like(parts, device="cpu").pin_memory()
        hp.copy_(parts)
        ht = torch.empty_like(temps, device="cpu").pin_memory()
        ht.copy_(temps)
        stride = 1 if temps.shape[0] == B else 0
        hws = torch.empty((plan.host_workspace_size(B, stride) + 256,), dtype=torch.uint8, device="cuda")
        hout = dict(euler=torch.empty((B, 3), dtype=torch.float64).pin_memory(),
                    R=torch.empty((B, 3, 3), dtype=torch.float64).pin_memory(),
                    score=torch.empty((B,), dtype=torch.float64).pin_memory(),
                    best_p=torch.empty((B,), dtype=torch.int32).pin_memory(),
                    flags=torch.empty((B,), dtype=torch.int32).pin_memory())
        m.matcha_align_host(plan, hp, ht, ws=hws, out=hout)
        ke = max(3, args.steps // 10)
        barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            m.matcha_align_host(plan, hp, ht, ws=hws, out=hout)
        te = (time.perf_counter() - t0) / ke
        te = max_over_ranks(te, ws, device="cuda")
        res["e2e"] = {"value": aggregate_rate(ws, B, te), "unit": UNIT,
                      "h2d_bytes_per_step": int(hp.numel() * 4 + ht.numel() * 4),
                      "d2h_bytes_per_step": int(B * (13 * 8 + 2 * 4)),
                      "api": "matcha_align_host (pinned host buffers, copies inside the call)"}
        del hws
    # further workloads, after the end-to-end measurement so that their device
    # allocations cannot affect it
    if rank == 0 and not args.no_backward:
        res["backward"] = time_backward(st)
    if rank == 0 and not args.no_mixed:
        res["mixed"] = time_mixed(st, prec)
        import torch
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_precision:
        res["precision"] = time_precision(st)
        import torch
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_study:
        res["refine_study"] = time_refine_study(st)
        import torch
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_pose6d:
        res["pose6d"] = time_pose6d(st, n=args.pose6d_batch)
        import torch
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_paper:
        res["paper_scale"] = time_paper_scale(st, n=args.paper_batch)
        import torch
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        cores = oracle.max_threads()
        nb = min(B, 5 * cores)
        kw = dict(S=w.n_shells, r_max=w.r_max, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter,
                  L_sched=w.L_sched)
        pc, tc = parts.cpu().numpy(), temps.cpu().numpy()
        t0 = time.perf_counter()
        ref = oracle.align_batch(pc[:nb], tc[:nb] if tc.shape[0] == B else tc, **kw)
        tcpu = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": nb / tcpu, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": "first %d particles of the batch, FP64 C oracle, %.1f s"
                                         % (nb, tcpu),
                               "cpu": host_cpu(),
                               "per_core": oracle_per_core(oracle, pc, tc, kw)}
        # the metric's accuracy gate: the oracle on every particle of the batch
        # (the rest of the batch, untimed), against every path's rotations
        if not args.no_oracle_gate and nb < B:
            rest = oracle.align_batch(pc[nb:], tc[nb:] if tc.shape[0] == B else tc, **kw)
            ref = {k: np.concatenate([ref[k], rest[k]]) for k in ref}
        if not args.no_oracle_gate:
            ties = oracle_near_ties(ref)
            res["accuracy"] = accuracy_vs_oracle(Rs, ref, d["R_true"].cpu().numpy()
                                                 if hasattr(d["R_true"], "cpu") else d["R_true"], ties)
            res["accuracy"]["oracle_seconds"] = time.perf_counter() - t0
    if rank == 0:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
