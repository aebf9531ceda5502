"""matcha_soft_search_noalloc against matcha_soft_search.

The allocation-free entry point serves callers that may not allocate device
memory themselves (device memory owned by one allocator or a fixed pool, or a
latency-critical loop where cudaMalloc's possible device synchronisation is
not acceptable).  It keeps the SOFFT grid in an array built into the library
instead of caller scratch.  Two calls in a row, on different inputs, must
give what the allocating entry point gives on the same inputs, and a batch
beyond the array's size must be refused with a clear error.

This file is collected last on purpose; it also passes on its own in a fresh
process.
"""
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


def _coeffs(plan, w, start):
    d = synth.make_batch(w, start=start)
    parts = d["particles"].cuda().contiguous()
    temps = d["templates"].cuda().contiguous()
    f = m.matcha_analyze(plan, parts)
    h = m.matcha_analyze(plan, temps)
    return m.matcha_correlate_coeffs(plan, f, h, 1)


@pytest.mark.parametrize("precision", [m.FP64, m.FP32], ids=["fp64", "fp32"])
def test_noalloc_matches_allocating_search_on_two_calls(precision):
    w = dataclasses.replace(synth.WORKLOADS["small32"], B=3)
    plan = m.plan_for_workload(w, precision=precision)
    B, P = w.B, w.P
    for call, start in enumerate((0, 3)):
        c = _coeffs(plan, w, start)
        ref = m.matcha_soft_search(plan, c)
        out = dict(idx=torch.full((B, P), 7, dtype=torch.int32, device="cuda"),
                   euler=torch.full((B, P, 3), 7.0, dtype=torch.float64, device="cuda"),
                   score=torch.full((B, P), 7.0, dtype=torch.float64, device="cuda"),
                   n_cand=torch.full((B,), 7, dtype=torch.int32, device="cuda"))
        got = m.matcha_soft_search_noalloc(plan, c, **out)
        torch.cuda.synchronize()
        assert torch.equal(got["n_cand"], ref["n_cand"]), call
        assert torch.equal(got["idx"], ref["idx"]), call
        for b in range(B):
            k = int(ref["n_cand"][b])
            assert torch.allclose(got["score"][b, :k], ref["score"][b, :k], rtol=1e-12, atol=0)
            assert torch.allclose(got["euler"][b, :k], ref["euler"][b, :k], rtol=0, atol=1e-15)


def test_noalloc_refuses_batches_beyond_the_builtin_array():
    w = synth.WORKLOADS["batch64"]
    plan = m.plan_for_workload(w, precision=m.FP64)
    n = plan.info.soft_n
    limit = (64 << 20) // (n ** 3 * 8)
    B = limit + 1
    c = torch.zeros((B, plan.info.corr_entries, 2, 2), dtype=torch.float64, device="cuda")
    outs = dict(idx=torch.empty((B, w.P), dtype=torch.int32, device="cuda"),
                euler=torch.empty((B, w.P, 3), dtype=torch.float64, device="cuda"),
                score=torch.empty((B, w.P), dtype=torch.float64, device="cuda"),
                n_cand=torch.empty((B,), dtype=torch.int32, device="cuda"))
    with pytest.raises(m.MatchaError, match="at most %d particles" % limit):
        m.matcha_soft_search_noalloc(plan, c, **outs)
