"""The ball-harmonic radial basis with the eigenvalue cut (Appendix "Ball
harmonics expansion and eigenvalue-based truncation"; Eq. sigmalmm through
the rank-|K_l| factors of Appendix "Low-rank structure induced by radial
sparsity") against the oracle: the correlation coefficients element by
element, the whole path in FP64 (1e-8 rad) and FP32 (0.05 degrees)."""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_15285_gb300 as m
import synth
from gpu_helpers import corr_to_oracle
from oracle import ball

pytestmark = pytest.mark.gpu
W = dataclasses.replace(synth.WORKLOADS["small32"], B=2)
LAM = 20.0


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("prec,tol", [(m.FP64, 1e-12), (m.FP32, 2e-6)], ids=["fp64", "fp32"])
def test_ball_coefficients_match_oracle(prec, tol):
    d = synth.make_batch(W)
    plan = m.plan_for_workload(W, precision=prec, ball_lambda=LAM)
    f = m.matcha_analyze(plan, d["particles"].cuda())
    h = m.matcha_analyze(plan, d["templates"].cuda())
    c = m.matcha_correlate_coeffs(plan, f, h, 1)
    torch.cuda.synchronize()
    L, S, R = W.L_sched[-1], W.n_shells, W.r_max
    Wt, counts = ball.radial_table(S, R, L, LAM)
    for b in range(W.B):
        fo = ball.project(O.analyze_volume(d["particles"][b].numpy(), S, R, L), Wt)
        ho = ball.project(O.analyze_volume(d["templates"][b].numpy(), S, R, L), Wt)
        co = ball.correlate_ball(fo, ho, counts, L)
        got = corr_to_oracle(c[b], L)
        assert np.abs(got - co).max() <= tol * np.abs(co).max()
    plan.close()


def test_ball_path_matches_oracle():
    d = synth.make_batch(W)
    ref = ball.align_ball(d["particles"].numpy(), d["templates"].numpy(), S=W.n_shells, r_max=W.r_max,
                          Lam=LAM, L0=W.L0, K=W.K, P=W.P, M_iter=W.M_iter, L_sched=W.L_sched)
    for prec in (m.FP64, m.FP32):
        plan = m.plan_for_workload(W, precision=prec, ball_lambda=LAM)
        out = m.matcha_align(plan, d["particles"].cuda(), d["templates"].cuda())
        torch.cuda.synchronize()
        for b in range(W.B):
            err = O.rotation_angle(out["R"][b].cpu().numpy(), ref["R"][b])
            if prec == m.FP64:
                assert err < 1e-8
                assert abs(out["score"][b].item() - ref["score"][b]) <= 1e-10 * abs(ref["score"][b])
            else:
                assert math.degrees(err) < 0.05
        plan.close()


def test_ball_plan_limits():
    with pytest.raises(m.MatchaError, match="ball"):
        m.plan_for_workload(W, precision=m.TF32, ball_lambda=LAM)
    with pytest.raises(m.MatchaError, match="radial functions"):
        m.plan_for_workload(W, precision=m.FP64, ball_lambda=200.0)   # |K_0| > 12 shells
