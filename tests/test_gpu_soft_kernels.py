"""The SOFFT search kernels of the 32-bit plans are interchangeable tile
choices: the chunked kernel, the warp-per-slice kernel and the register-tiled
kernel give bit-identical grids, candidates and refined results (FP32 and TF32
plans, fixed and per-particle candidate counts), and the autotuner may pick
any of them."""
import dataclasses

import pytest
import torch

import paper_2603_15285_gb300 as m
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name,prec", [("batch64", m.FP32), ("batch64", m.TF32), ("var48", m.FP32),
                                       ("small32", m.FP32)],
                         ids=["batch64_fp32", "batch64_tf32", "var48_fp32", "small32_fp32"])
def test_soft_kernels_bit_identical(name, prec):
    w = dataclasses.replace(synth.WORKLOADS[name], B=96 if name != "small32" else 1)
    d = synth.make_batch(w, device="cuda")
    P_per = torch.from_numpy(d["P_per"]).cuda() if w.P_range else None
    plan = m.plan_for_workload(w, precision=prec)
    f = m.matcha_analyze(plan, d["particles"])
    h = m.matcha_analyze(plan, d["templates"])
    c = m.matcha_correlate_coeffs(plan, f, h, 1)
    outs = []
    for k in (1, 2, 3):
        plan.set_tiles(soft_kernel=k)
        soft = m.matcha_soft_search(plan, c, P_per=P_per)
        al = m.matcha_align(plan, d["particles"], d["templates"], P_per=P_per)
        torch.cuda.synchronize()
        outs.append((soft, al))
    same = lambda a, b: torch.testing.assert_close(a, b, rtol=0, atol=0, equal_nan=True)
    s1, a1 = outs[0]
    for s2, a2 in outs[1:]:
        for key in ("grid", "idx", "score", "euler", "n_cand"):   # scores past n_cand are NaN
            same(s1[key], s2[key])
        for key in ("euler", "R", "score", "best_p", "flags"):
            same(a1[key], a2[key])
    plan.close()


def test_autotuner_reports_the_soft_kernel():
    w = dataclasses.replace(synth.WORKLOADS["batch64"], B=256)
    d = synth.make_batch(w, device="cuda")
    plan = m.plan_for_workload(w, precision=m.FP32)
    rep = plan.autotune(d["particles"], d["templates"])
    print("autotune:", rep)
    assert rep["soft_kernel"] in (1, 2, 3) and min(rep["soft_ms"]) > 0
    plan64 = m.plan_for_workload(w, precision=m.FP64)
    with pytest.raises(m.MatchaError):
        plan64.set_tiles(soft_kernel=2)     # the warp kernel serves the 32-bit plans only
    with pytest.raises(m.MatchaError):
        plan64.set_tiles(soft_kernel=3)     # so does the register-tiled kernel


@pytest.mark.parametrize("name,prec,B", [("var48", m.FP32, 200), ("batch64", m.FP32, 300),
                                         ("batch64", m.FP64, 40)],
                         ids=["var48_fp32", "batch64_fp32_parts", "batch64_fp64"])
def test_newton_schedules_bit_identical(name, prec, B):
    """One CTA per particle in index order, and persistent CTAs pulling particles
    from the queue sorted by decreasing candidate count: the same results bit for
    bit (each particle's arithmetic does not depend on which CTA runs it)."""
    w = dataclasses.replace(synth.WORKLOADS[name], B=B)
    d = synth.make_batch(w, device="cuda")
    P_per = torch.from_numpy(d["P_per"]).cuda() if w.P_range else None
    plan = m.plan_for_workload(w, precision=prec)
    outs = []
    for k in (1, 2):
        plan.set_tiles(newton_sched=k)
        outs.append(m.matcha_align(plan, d["particles"], d["templates"], P_per=P_per))
        torch.cuda.synchronize()
    for key in ("euler", "R", "score", "best_p", "flags"):
        torch.testing.assert_close(outs[0][key], outs[1][key], rtol=0, atol=0, equal_nan=True)
    rep = plan.autotune(d["particles"], d["templates"], P_per=P_per)
    print("%s: newton schedule times (ms) %s -> %d" % (name, rep["newton_ms"], rep["newton_sched"]))
    assert rep["newton_sched"] in (1, 2)
    plan.close()
