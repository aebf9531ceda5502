"""The contraction on the tensor cores (TF32 and BF16 operands, FP32
accumulation): elementwise against the oracle within the rounding bound of
the operands, and the whole path within 0.05 degrees of the FP64 path."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_15285_gb300 as m
import synth
from gpu_helpers import corr_to_oracle

pytestmark = pytest.mark.gpu
W = synth.WORKLOADS["batch64"]
# unit roundoff of the operands: TF32 keeps 10 fraction bits, BF16 7
UNIT = {m.TF32: 2.0 ** -11, m.BF16: 2.0 ** -8}


@pytest.fixture(scope="module")
def batch():
    import __graft_entry__
    __graft_entry__.build()
    return synth.make_batch(W, device="cuda")


@pytest.mark.parametrize("prec", [m.TF32, m.BF16])
def test_tc_contraction_within_operand_rounding_of_oracle(batch, prec):
    """|c_tc - c_oracle| <= 3u sum_s w_s |f_lm| |h_ln| + 1e-6 max|c|: each product
    of two operands rounded to u (2u + u^2), FP32 accumulation and the FP32
    analysis far below that."""
    B = 2
    parts = batch["particles"][:B].contiguous()
    temps = batch["templates"][:B].contiguous()
    plan = m.plan_for_workload(W, precision=prec)
    f = m.matcha_analyze(plan, parts)
    h = m.matcha_analyze(plan, temps)
    c = m.matcha_correlate_coeffs(plan, f, h, 1)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    S, R, L = W.n_shells, W.r_max, W.L_sched[-1]
    r, ws = O.radial_nodes(S, R)
    u = UNIT[prec]
    for b in range(B):
        fo = O.analyze_volume(parts[b].cpu().numpy(), S, R, L)
        ho = O.analyze_volume(temps[b].cpu().numpy(), S, R, L)
        co = O.correlate(fo, ho, S, R, L)
        cg = corr_to_oracle(c[b], L)
        # sum_s w_s |f_lm| |h_ln| over the full (l, m, n) layout
        af, ah = np.abs(fo), np.abs(ho)
        bound = np.zeros(O.c_size(L))
        for l in range(L + 1):
            for mm in range(-l, l + 1):
                fm = af[:, O.lm_index(l, abs(mm))]
                for nn in range(-l, l + 1):
                    bound[O.c_index(l, mm, nn)] = np.sum(ws * fm * ah[:, O.lm_index(l, abs(nn))])
        tol = 3 * u * bound + 1e-6 * np.abs(co).max()
        err = np.abs(cg - co)
        print("tc contraction (%s) particle %d: max err/bound %.3f, max rel %.2e"
              % ("tf32" if prec == m.TF32 else "bf16", b, (err / tol).max(),
                 err.max() / np.abs(co).max()))
        assert np.all(err <= tol)
    plan.close()


@pytest.fixture(scope="module")
def fp64_R(batch):
    plan = m.plan_for_workload(W, precision=m.FP64)
    out = m.matcha_align(plan, batch["particles"], batch["templates"])
    torch.cuda.synchronize()
    plan.close()
    return out["R"].cpu().numpy()


@pytest.mark.parametrize("prec", [m.TF32, m.BF16])
def test_tc_path_within_005_degrees_of_fp64(batch, fp64_R, prec):
    plan = m.plan_for_workload(W, precision=prec)
    out = m.matcha_align(plan, batch["particles"], batch["templates"])
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    R = out["R"].cpu().numpy()
    errs = np.degrees([O.rotation_angle(R[b], fp64_R[b]) for b in range(R.shape[0])])
    print("%s path vs FP64 (1024 particles): max %.3e deg, p90 %.3e deg"
          % ("tf32" if prec == m.TF32 else "bf16", errs.max(), np.percentile(errs, 90)))
    assert errs.max() < 0.05
    plan.close()


def test_tc_plan_rejects_bandwidth_64():
    with pytest.raises(m.MatchaError):
        m.Plan(box_n=64, n_shells=32, L0=8, K=2, P=16, M_iter=3, L_sched=[8, 64], precision=m.TF32)


def test_forced_wait_timeout_sets_status_and_recovers(batch):
    """With a wait limit of 0 polls every CTA gives up on its first MMA wait:
    the status word reports it (and is cleared by the read), the CTAs drain
    their MMAs and free their tensor memory, and the next call with the
    built-in limit is correct again."""
    B = 8
    parts = batch["particles"][:B].contiguous()
    temps = batch["templates"][:B].contiguous()
    plan = m.plan_for_workload(W, precision=m.TF32)
    f = m.matcha_analyze(plan, parts)
    h = m.matcha_analyze(plan, temps)
    good = m.matcha_correlate_coeffs(plan, f, h, 1)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    plan.set_wait_limit(0)
    m.matcha_correlate_coeffs(plan, f, h, 1)
    torch.cuda.synchronize()
    assert plan.device_status() == 1
    assert plan.device_status() == 0  # cleared by the read
    plan.set_wait_limit(-1)
    again = m.matcha_correlate_coeffs(plan, f, h, 1)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    assert torch.equal(again, good)
    plan.close()
