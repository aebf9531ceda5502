"""Host-side helpers of bench.py: the per-kernel roofline arithmetic, the L2
note, the kernel count of a step and the CPU-baseline helpers (no GPU needed)."""
import math

import bench
import paper_2603_15285_gb300 as m
import synth


def test_l2_note_compares_with_129_mb():
    assert "> 129 MB L2" in bench.l2_note(2 * 1024 * 64 ** 3 * 4)
    assert "below the 129 MB L2" in bench.l2_note(2 * 8 * 64 ** 3 * 4)


def test_kernel_roofline_arithmetic():
    w = synth.WORKLOADS["batch64"]
    B = 1024
    st = dict(analyze=2.0, correlate=0.5, soft=1.0, newton=2.0, select=0.01)
    r = bench.kernel_roofline(w, B, m.FP32, st, 80.0, m)
    peaks = bench.measured_peaks()
    # analysis: particle + template volumes, 4 bytes per voxel, once each
    want = 2 * 4 * 64 ** 3 * B / 2e-3 / 1e9
    assert math.isclose(r["analysis"]["achieved"], want, rel_tol=1e-12)
    assert math.isclose(r["analysis"]["frac"], want / peaks["hbm_gbs"], rel_tol=1e-12)
    # and in flops: 32 shells x (33 rings x 66 samples x 33 orders + 561 (l, m) x 33 nodes)
    # complex multiply-adds of 4 flops, two volumes: 23.1 MFLOP per particle
    assert r["analysis"]["flops_per_particle"] == 2 * 32 * 4 * (33 * 66 * 33 + 561 * 33)
    assert math.isclose(r["analysis"]["alu_frac"],
                        r["analysis"]["flops_per_particle"] * B / 2e-3 / 1e12 / 80.0, rel_tol=1e-12)
    # contraction: 8 S T(L) flops per particle, T(32) = 47,905
    T = 33 * 65 * 67 // 3
    assert T == 47905
    assert math.isclose(r["contraction"]["achieved"], 8.0 * 32 * T * B / 0.5e-3 / 1e12, rel_tol=1e-12)
    assert math.isclose(r["contraction"]["frac"], r["contraction"]["achieved"] / 80.0, rel_tol=1e-12)
    assert math.isclose(r["soft"]["grid_points_per_s"], 36 ** 3 * B / 1e-3, rel_tol=1e-12)
    # tensor-core plans are measured against the tensor peak of their operand type
    r16 = bench.kernel_roofline(w, B, m.BF16, st, 80.0, m)
    r32 = bench.kernel_roofline(w, B, m.TF32, st, 80.0, m)
    assert r16["contraction"]["bound"] == "tensor"
    assert math.isclose(r32["contraction"]["peak"], r16["contraction"]["peak"] * 1.1 / 2.25,
                        rel_tol=1e-12)


def test_cpu_baseline_per_core_and_host_model():
    import oracle
    assert isinstance(bench.host_cpu(), str) and bench.host_cpu()
    w = synth.WORKLOADS["small32"]
    d = synth.make_batch(w, B=2)
    kw = dict(S=w.n_shells, r_max=w.r_max, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter,
              L_sched=w.L_sched)
    r = bench.oracle_per_core(oracle, d["particles"].numpy(), d["templates"].numpy(), kw, n=1)
    assert r["cores"] == 1 and r["value"] > 0 and "one thread" in r["sample"]


def test_wigner_term_units_of_the_bench_workload():
    w = synth.WORKLOADS["batch64"]
    r = bench.wigner_term_units(w, 1024, 2.0, 80.0)
    # 3 P sum_j T(L_j), T(L) = (L+1)(2L+1)(2L+3)/3, L = 8, 16, 24, 32, P = 16
    assert r["wigner_terms_per_particle"] == 3 * 16 * (969 + 6545 + 20825 + 47905) == 3659712
    assert math.isclose(r["achieved"], 30.0 * 3659712 * 1024 / 2e-3 / 1e12, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / 80.0, rel_tol=1e-12)
