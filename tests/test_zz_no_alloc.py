"""matcha_soft_search_noalloc against matcha_soft_search.

The allocation-free entry point serves callers that may not allocate device
memory themselves (device memory owned by one allocator or a fixed pool, or a
latency-critical loop where cudaMalloc's possible device synchronisation is
not acceptable).  Plans whose SOFFT grid goes through memory keep it in an
array built into the library instead of caller scratch; plans whose grid
stays on chip need no scratch.  Two calls in a row, on different inputs, must
give what the allocating entry point gives on the same inputs, on both kinds
of plan, and a batch beyond the array's size must be refused with a clear
error.

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


def _outputs(B, P):
    return dict(idx=torch.full((B, P), 7, dtype=torch.int32, device="cuda"),
                euler=torch.full((B, P, 3), 7.0, dtype=torch.float64, device="cuda"),
                score=torch.full((B, P), 7.0, dtype=torch.float64, device="cuda"),
                n_cand=torch.full((B,), 7, dtype=torch.int32, device="cuda"))


def _same(got, ref, B, exact):
    assert torch.equal(got["n_cand"], ref["n_cand"])
    assert torch.equal(got["idx"], ref["idx"])
    for b in range(B):
        k = int(ref["n_cand"][b])
        if exact:
            assert torch.equal(got["score"][b, :k], ref["score"][b, :k])
            assert torch.equal(got["euler"][b, :k], ref["euler"][b, :k])
        else:
            assert torch.allclose(got["score"][b, :k], ref["score"][b, :k], rtol=1e-12, atol=0)
            assert torch.allclose(got["euler"][b, :k], ref["euler"][b, :k], rtol=0, atol=1e-15)


@pytest.mark.parametrize("precision", [m.FP64, m.FP32], ids=["fp64", "fp32"])
def test_noalloc_matches_allocating_search_on_two_calls(precision):
    """A plan whose SOFFT grid stays on chip (L0 = 8): no scratch is used."""
    w = dataclasses.replace(synth.WORKLOADS["small32"], B=3)
    plan = m.plan_for_workload(w, precision=precision)
    B, P = w.B, w.P
    for call, start in enumerate((0, 3)):
        c = _coeffs(plan, w, start)
        ref = m.matcha_soft_search(plan, c)
        got = m.matcha_soft_search_noalloc(plan, c, **_outputs(B, P))
        torch.cuda.synchronize()
        _same(got, ref, B, exact=False)


@pytest.mark.parametrize("precision", [m.FP64, m.FP32], ids=["fp64", "fp32"])
def test_noalloc_grid_in_builtin_array_on_two_calls(precision):
    """A plan whose SOFFT grid goes through memory (L0 = 30, K = 2: 124^3 points
    per particle): the grid lives in the library's array.  Two calls in a row on
    different coefficients equal the allocating search bit for bit."""
    w = synth.WORKLOADS["paper200"]
    plan = m.plan_for_workload(w, precision=precision)
    n, B, P = plan.info.soft_n, 2, w.P
    gen = torch.Generator(device="cpu").manual_seed(5)
    shape = (B, plan.info.corr_entries, 2, 2)
    # this plan materialises the grid: the allocating search overwrites a NaN grid
    c = torch.randn(shape, generator=gen, dtype=torch.float64).to(plan.real_dtype).cuda()
    grid = torch.full((B, n, n, n), float("nan"), dtype=plan.real_dtype, device="cuda")
    m.matcha_soft_search(plan, c, grid=grid)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(grid).all())
    for call in range(2):
        c = torch.randn(shape, generator=gen, dtype=torch.float64).to(plan.real_dtype).cuda()
        ref = m.matcha_soft_search(plan, c)
        got = m.matcha_soft_search_noalloc(plan, c, **_outputs(B, P))
        torch.cuda.synchronize()
        assert int(ref["n_cand"].min()) > 0, call
        _same(got, ref, B, exact=True)


def test_noalloc_refuses_batches_beyond_the_builtin_array():
    w = synth.WORKLOADS["paper200"]
    plan = m.plan_for_workload(w, precision=m.FP64)
    n = plan.info.soft_n
    limit = (64 << 20) // (n ** 3 * 8)
    B = limit + 1
    c = torch.zeros((B, plan.info.corr_entries, 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(m.MatchaError, match="at most %d particles" % limit):
        m.matcha_soft_search_noalloc(plan, c, **_outputs(B, w.P))


def test_noalloc_on_chip_plan_has_no_scratch_limit():
    """The 64^3 plan (L0 = 8) keeps its grid on chip: a batch far beyond what the
    array could hold as a grid is served and equals the allocating search."""
    w = synth.WORKLOADS["batch64"]
    plan = m.plan_for_workload(w, precision=m.FP64)
    n = plan.info.soft_n
    B = (64 << 20) // (n ** 3 * 8) + 21
    gen = torch.Generator(device="cpu").manual_seed(9)
    c = torch.randn((B, plan.info.corr_entries, 2, 2), generator=gen, dtype=torch.float64).cuda()
    ref = m.matcha_soft_search(plan, c)
    got = m.matcha_soft_search_noalloc(plan, c, **_outputs(B, w.P))
    torch.cuda.synchronize()
    _same(got, ref, B, exact=True)
