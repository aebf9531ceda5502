"""The analysis reads the trilinear corners through 2x2 texture gathers when a
batch qualifies (row pitch and base alignment) and through plain loads
otherwise; both must give the same coefficients bit for bit, in both plan
precisions.  A copy of the batch at a 4-byte offset misses the texture base
alignment and takes the load path."""
import dataclasses

import numpy as np
import pytest
import torch

import paper_2603_15285_gb300 as m
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name,prec", [("small32", m.FP64), ("small32", m.FP32),
                                       ("batch64", m.FP32), ("batch64", m.FP64)],
                         ids=["small32_fp64", "small32_fp32", "batch64_fp32", "batch64_fp64"])
def test_texture_and_load_paths_agree(name, prec):
    w = dataclasses.replace(synth.WORKLOADS[name], B=3)
    d = synth.make_batch(w)
    vols = d["particles"].cuda().contiguous()
    plan = m.plan_for_workload(w, precision=prec)
    tex = m.matcha_analyze(plan, vols)
    # the same voxels one float past a 512-byte boundary: no texture view
    buf = torch.empty(vols.numel() + 1, dtype=torch.float32, device="cuda")
    shifted = buf[1:].view_as(vols)
    shifted.copy_(vols)
    assert shifted.data_ptr() % 512 != 0
    ld = m.matcha_analyze(plan, shifted)
    torch.cuda.synchronize()
    assert torch.equal(tex, ld)
    plan.close()


@pytest.mark.parametrize("prec", [m.FP64, m.FP32], ids=["fp64", "fp32"])
def test_shells_beyond_the_box(prec):
    """Outer shells of radius up to 0.7 N leave the box: their samples are the
    zero-padded trilinear values (bounds-checked path) on both read paths, and
    the FP64 coefficients match the oracle's analysis."""
    w = dataclasses.replace(synth.WORKLOADS["small32"], B=2)
    d = synth.make_batch(w)
    vols = d["particles"].cuda().contiguous()
    R = 0.7 * w.N
    plan = m.Plan(box_n=w.N, n_shells=w.n_shells, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter,
                  L_sched=w.L_sched, precision=prec, r_max=R)
    tex = m.matcha_analyze(plan, vols)
    buf = torch.empty(vols.numel() + 1, dtype=torch.float32, device="cuda")
    shifted = buf[1:].view_as(vols)
    shifted.copy_(vols)
    ld = m.matcha_analyze(plan, shifted)
    torch.cuda.synchronize()
    assert torch.equal(tex, ld)
    if prec == m.FP64:
        import oracle as O
        from gpu_helpers import coef_to_complex
        f = coef_to_complex(tex)
        for b in range(vols.shape[0]):
            ref = O.analyze_volume(d["particles"][b].numpy(), w.n_shells, R, w.L_final)
            assert np.abs(f[b] - ref).max() <= 1e-12 * np.abs(ref).max()
    plan.close()
