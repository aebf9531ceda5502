"""The analysis reads the trilinear corners through 2x2 texture gathers when a
batch qualifies (row pitch and base alignment) and through plain loads
otherwise; both must give the same coefficients bit for bit, in both plan
precisions.  A copy of the batch at a 4-byte offset misses the texture base
alignment and takes the load path."""
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
