"""Section 5.1's comparisons on the GPU: refinement by gradient steps instead
of Newton steps (same step control), against the oracle's gradient march, and
the dense SOFFT baseline at high oversampling (K = 8, 16: grids through HBM)
against the oracle's grid and candidate selection."""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_15285_gb300 as m
import synth
from gpu_helpers import oracle_align

pytestmark = pytest.mark.gpu
W = synth.WORKLOADS["small32"]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("M", [3, 12])
def test_gradient_refinement_matches_oracle(M):
    w = dataclasses.replace(W, M_iter=M)
    d = synth.make_batch(w)
    ref = oracle_align(w, d["particles"].numpy(), d["templates"].numpy(), refine=1)
    plan = m.plan_for_workload(w, precision=m.FP64, refine=1)
    out = m.matcha_align(plan, d["particles"].cuda(), d["templates"].cuda())
    torch.cuda.synchronize()
    err = O.rotation_angle(out["R"][0].cpu().numpy(), ref["R"][0])
    assert err < 1e-8
    assert abs(out["score"][0].item() - ref["score"][0]) <= 1e-10 * abs(ref["score"][0])
    assert int(out["flags"][0]) & 2 == 0
    plan.close()


def test_gradient_needs_more_steps_than_newton():
    d = synth.make_batch(W)
    ref = oracle_align(W, d["particles"].numpy(), d["templates"].numpy())
    errs = {}
    for refine in (0, 1):
        plan = m.plan_for_workload(W, precision=m.FP64, refine=refine)
        out = m.matcha_align(plan, d["particles"].cuda(), d["templates"].cuda())
        torch.cuda.synchronize()
        errs[refine] = O.rotation_angle(out["R"][0].cpu().numpy(), ref["R"][0])
        plan.close()
    assert errs[0] < 1e-8 and errs[1] > 10 * errs[0]


def test_dense_soft_grid_and_candidates_match_oracle_at_k8():
    w = dataclasses.replace(W, K=8)
    d = synth.make_batch(w)
    plan = m.plan_for_workload(w, precision=m.FP64)
    f = m.matcha_analyze(plan, d["particles"].cuda())
    h = m.matcha_analyze(plan, d["templates"].cuda())
    c = m.matcha_correlate_coeffs(plan, f, h, 1)
    soft = m.matcha_soft_search(plan, c)
    torch.cuda.synchronize()
    L0, S, R, L = w.L0, w.n_shells, w.r_max, w.L_sched[-1]
    fo = O.analyze_volume(d["particles"][0].numpy(), S, R, L)     # the plan's angular grid
    ho = O.analyze_volume(d["templates"][0].numpy(), S, R, L)
    co = O.correlate(fo, ho, S, R, L)
    grid = O.soft_grid(co, L0, w.K)
    n = O.soft_n(L0, w.K)
    assert n == 144
    g = soft["grid"][0].cpu().numpy().reshape(-1)
    assert np.abs(g - grid).max() <= 1e-10 * np.abs(grid).max()
    idx, sc = O.local_maxima_topk(grid, n, w.P)
    k = int(soft["n_cand"][0])
    assert list(soft["idx"][0, :k].cpu().numpy()) == list(idx)
    plan.close()


def test_dense_soft_k16_best_point_near_refined_rotation():
    """K = 16 (288 points per angle, 24 M per particle): the grid's best point
    lies within one grid step of the refined rotation."""
    w = dataclasses.replace(W, K=16)
    d = synth.make_batch(w)
    plan = m.plan_for_workload(w, precision=m.FP32)
    f = m.matcha_analyze(plan, d["particles"].cuda())
    h = m.matcha_analyze(plan, d["templates"].cuda())
    c = m.matcha_correlate_coeffs(plan, f, h, 1)
    soft = m.matcha_soft_search(plan, c)
    torch.cuda.synchronize()
    ref = oracle_align(W, d["particles"].numpy(), d["templates"].numpy())
    eu = soft["euler"][0, 0].cpu().numpy()
    step = 2 * math.pi / O.soft_n(w.L0, w.K)
    err = O.rotation_angle(O.euler_to_matrix(*eu), ref["R"][0])
    assert err < 2 * step
    plan.close()
