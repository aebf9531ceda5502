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
