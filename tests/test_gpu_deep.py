"""The 64^3 workload marched to bandwidth 48 (schedule 8 -> 16 -> ... -> 48,
three Newton steps per level): FP64 results against the oracle on a sample,
FP32 results against the FP64 GPU results (0.05 degrees) on a batch.  At this
bandwidth the refinement kernel holds fewer staging buffers and the analysis
kernel one shell per block in FP64; both paths are exercised here."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_15285_gb300 as m
import synth
from gpu_helpers import oracle_align

pytestmark = pytest.mark.gpu
W = synth.WORKLOADS["deep64"]
B = 256
SAMPLE = [0, 255]


@pytest.fixture(scope="module")
def batch():
    import __graft_entry__
    __graft_entry__.build()
    return synth.make_batch(W, B=B, device="cuda")


@pytest.fixture(scope="module")
def fp64_result(batch):
    plan = m.plan_for_workload(W, precision=m.FP64)
    out = m.matcha_align(plan, batch["particles"], batch["templates"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_deep_fp64_matches_oracle_on_sample(batch, fp64_result):
    parts = batch["particles"][SAMPLE].cpu().numpy()
    temps = batch["templates"][SAMPLE].cpu().numpy()
    ref = oracle_align(W, parts, temps)
    for i, b in enumerate(SAMPLE):
        assert O.rotation_angle(fp64_result["R"][b], ref["R"][i]) < 1e-8
        assert abs(fp64_result["score"][b] - ref["score"][i]) <= 1e-10 * abs(ref["score"][i])


def test_deep_fp32_within_005_degrees(batch, fp64_result):
    plan = m.plan_for_workload(W, precision=m.FP32)
    out = m.matcha_align(plan, batch["particles"], batch["templates"])
    R = out["R"].cpu().numpy()
    errs = np.array([O.rotation_angle(R[b], fp64_result["R"][b]) for b in range(B)])
    print("deep64 fp32 vs fp64 GPU: max %.3e deg" % math.degrees(errs.max()))
    assert math.degrees(errs.max()) < 0.05
    assert np.all(np.isfinite(out["score"].cpu().numpy()))


def test_max_bandwidth_64_fp64_matches_oracle_and_fp32_within_005():
    """L_J = 64, the library's limit (schedule 8 -> 16 -> 32 -> 64): FP64 against
    the oracle on one particle, FP32 within 0.05 degrees of FP64 on the batch."""
    w = synth.WORKLOADS["max64"]
    d = synth.make_batch(w, device="cuda")
    parts, temps = d["particles"].contiguous(), d["templates"].contiguous()
    p64 = m.plan_for_workload(w, precision=m.FP64)
    o64 = m.matcha_align(p64, parts, temps)
    p32 = m.plan_for_workload(w, precision=m.FP32)
    o32 = m.matcha_align(p32, parts, temps)
    torch.cuda.synchronize()
    R64, R32 = o64["R"].cpu().numpy(), o32["R"].cpu().numpy()
    ref = oracle_align(w, parts[:1].cpu().numpy(), temps[:1].cpu().numpy())
    assert O.rotation_angle(R64[0], ref["R"][0]) < 1e-8
    assert abs(o64["score"][0].item() - ref["score"][0]) <= 1e-10 * abs(ref["score"][0])
    errs = np.degrees([O.rotation_angle(R32[b], R64[b]) for b in range(w.B)])
    print("max64: fp32 vs fp64 max %.3e deg" % errs.max())
    assert errs.max() < 0.05


@pytest.mark.parametrize("prec", [m.FP64, m.FP32])
def test_zero_volumes_are_degenerate_not_fatal(prec):
    """All-zero particle and template: C vanishes everywhere, every grid point
    ties, the Hessian is zero (gradient fallback with a zero step): the call
    returns, with finite outputs and the ties broken by index."""
    w = synth.WORKLOADS["small32"]
    z = torch.zeros((2, w.N, w.N, w.N), dtype=torch.float32, device="cuda")
    plan = m.plan_for_workload(w, precision=prec)
    out = m.matcha_align(plan, z, z)
    torch.cuda.synchronize()
    assert torch.all(out["score"] == 0)
    assert torch.all(torch.isfinite(out["euler"]))
    assert torch.all(out["best_p"] == 0)
