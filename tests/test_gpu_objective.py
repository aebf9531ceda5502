"""matcha_objective: C_L, its gradient and Hessian (Section 2.2) at given
rotations, against the oracle's objective on the oracle's own coefficients:
FP64 at 1e-10 of the scale, the 32-bit plans within their rounding level,
including the per-degree rescaled recurrence at L = 100."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_15285_gb300 as m
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name,prec,tol", [("small32", m.FP64, 1e-10), ("batch64", m.FP32, 2e-5),
                                           ("wide64", m.FP32, 2e-4), ("wide64", m.FP64, 1e-10)],
                         ids=["small32_fp64", "batch64_fp32", "wide64_fp32", "wide64_fp64"])
def test_objective_matches_oracle(name, prec, tol):
    w = synth.WORKLOADS[name]
    d = synth.make_batch(w, B=1)
    plan = m.plan_for_workload(w, precision=prec)
    f = m.matcha_analyze(plan, d["particles"].cuda())
    h = m.matcha_analyze(plan, d["templates"].cuda())
    c = m.matcha_correlate_coeffs(plan, f, h, 1)
    rng = np.random.default_rng(12)
    Q = min(plan.P, 8)
    pts = np.stack([rng.uniform(0, 2 * np.pi, Q), rng.uniform(0.02, np.pi - 0.02, Q),
                    rng.uniform(0, 2 * np.pi, Q)], axis=1)[None]
    L, S, R = w.L_sched[-1], w.n_shells, w.r_max
    fo = O.analyze_volume(d["particles"][0].numpy(), S, R, L)
    ho = O.analyze_volume(d["templates"][0].numpy(), S, R, L)
    co = O.correlate(fo, ho, S, R, L)
    for Lq in sorted({w.L_sched[0], L}):
        got = m.matcha_objective(plan, c, torch.from_numpy(pts).cuda(), L=Lq).cpu().numpy()[0]
        for q in range(Q):
            C, g, H, _ = O.objective(co, Lq, *pts[0, q], derivs=True)
            ref = np.array([C, *g, H[0, 0], H[0, 1], H[0, 2], H[1, 1], H[1, 2], H[2, 2]])
            scale = np.abs(ref).max()
            err = np.abs(got[q] - ref).max() / scale
            assert err < tol, (Lq, q, err)
    plan.close()


@pytest.mark.parametrize("name,prec", [("small32", m.FP64), ("batch64", m.FP64), ("batch64", m.FP32)],
                         ids=["small32_fp64", "batch64_fp64", "batch64_fp32"])
def test_objective_near_the_poles(name, prec):
    """Points within 1e-4 .. 1e-2 rad of beta = 0 and beta = pi, where the
    differential equation that gives d'' divides by sin^2(beta): FP64 keeps
    every component within 1e-10 of the oracle (relative to the largest); in
    FP32 the value and gradient stay within 2e-5 everywhere and the Hessian
    within 2e-5 from 1e-2 rad of a pole on (closer in it loses digits as
    u / sin^2 b, which only shapes the step direction)."""
    w = synth.WORKLOADS[name]
    d = synth.make_batch(w, B=1)
    plan = m.plan_for_workload(w, precision=prec)
    f = m.matcha_analyze(plan, d["particles"].cuda())
    h = m.matcha_analyze(plan, d["templates"].cuda())
    c = m.matcha_correlate_coeffs(plan, f, h, 1)
    betas = np.array([1e-4, 1e-3, 1e-2, np.pi - 1e-2, np.pi - 1e-3, np.pi - 1e-4])
    rng = np.random.default_rng(3)
    Q = len(betas)
    pts = np.stack([rng.uniform(0, 2 * np.pi, Q), betas, rng.uniform(0, 2 * np.pi, Q)], axis=1)[None]
    L, S, R = w.L_sched[-1], w.n_shells, w.r_max
    co = O.correlate(O.analyze_volume(d["particles"][0].numpy(), S, R, L),
                     O.analyze_volume(d["templates"][0].numpy(), S, R, L), S, R, L)
    got = m.matcha_objective(plan, c, torch.from_numpy(np.ascontiguousarray(pts)).cuda(),
                             L=L).cpu().numpy()[0]
    for q in range(Q):
        C, g, H, _ = O.objective(co, L, *pts[0, q], derivs=True)
        ref = np.array([C, *g, H[0, 0], H[0, 1], H[0, 2], H[1, 1], H[1, 2], H[2, 2]])
        err = np.abs(got[q] - ref) / np.abs(ref).max()
        if prec == m.FP64:
            assert err.max() < 1e-10, (q, err)
        else:
            assert err[:4].max() < 2e-5, (q, err)
            s = np.sin(betas[q])
            if s >= np.sin(1e-2) * 0.999:
                assert err[4:].max() < 2e-5, (q, err)
    plan.close()
