"""6-D pose (rotation and translation) against the oracle: the volume pose
transform, the translation search at a fixed rotation and the alternation of
the rotation search with the translation search (the appendix "Alternating
search over rotations and translations")."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_15285_gb300 as m
import synth
from oracle import translation as T

pytestmark = pytest.mark.gpu
W32 = synth.WORKLOADS["shift32"]
W64 = synth.WORKLOADS["shift64"]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_transform_volumes_fp64_equals_oracle_bit_for_bit():
    rng = np.random.default_rng(4)
    N, B = 24, 3
    vol = rng.standard_normal((B, N, N, N)).astype(np.float32)
    Rs = np.stack([synth.haar_rotation(rng) for _ in range(B)])
    sh = rng.uniform(-3, 3, size=(B, 3))
    got = m.matcha_transform_volumes(torch.from_numpy(vol).cuda(), torch.from_numpy(Rs).cuda(),
                                     torch.from_numpy(sh).cuda(), precision=m.FP64).cpu().numpy()
    got32 = m.matcha_transform_volumes(torch.from_numpy(vol).cuda(), torch.from_numpy(Rs).cuda(),
                                       torch.from_numpy(sh).cuda(), precision=m.FP32).cpu().numpy()
    for b in range(B):
        ref = T.transform_volume(vol[b], Rs[b], sh[b])
        assert np.array_equal(got[b], ref), b
        assert np.abs(got32[b] - ref).max() <= 1e-5 * np.abs(ref).max()
    # one shared input volume, identity rotation, shift only
    got = m.matcha_transform_volumes(torch.from_numpy(vol[:1]).cuda(), None,
                                     torch.from_numpy(sh).cuda(), B=B, precision=m.FP64).cpu().numpy()
    for b in range(B):
        assert np.array_equal(got[b], T.transform_volume(vol[0], None, sh[b]))


@pytest.mark.parametrize("w,upsample", [(W32, 10), (W32, 1), (W64, 10)], ids=["32_U10", "32_U1", "64_U10"])
def test_shift_search_matches_oracle(w, upsample):
    B = 2
    d = synth.make_batch(w, B=B)
    parts = d["particles"]
    Rt = torch.from_numpy(d["R_true"])
    rot = m.matcha_transform_volumes(d["templates"].cuda(), Rt.cuda(), precision=m.FP64)
    rot_h = rot.cpu().numpy()
    for prec in (m.FP64, m.FP32):
        plan = m.plan_for_workload(w, precision=prec)
        out = m.matcha_shift_search(plan, parts.cuda(), rot, w.max_shift, upsample, R=Rt.cuda())
        torch.cuda.synchronize()
        for b in range(B):
            t, cc, fl = T.shift_search(parts[b].numpy(), rot_h[b], w.max_shift, upsample)
            got_t = out["t"][b].cpu().numpy()
            if prec == m.FP64:
                assert np.array_equal(got_t, t), (b, got_t, t)
                assert abs(out["cc"][b].item() - cc) <= 1e-10 * abs(cc)
            else:
                assert np.abs(got_t - t).max() <= 1.0 / upsample + 1e-12, (b, got_t, t)
                assert abs(out["cc"][b].item() - cc) <= 1e-4 * abs(cc)
            assert int(out["flags"][b]) == fl
            tau = out["tau"][b].cpu().numpy()
            assert np.allclose(tau, d["R_true"][b].T @ got_t, atol=1e-12)
        plan.close()


def test_align6d_fp64_matches_oracle_and_fp32_close():
    w = W32
    d = synth.make_batch(w)
    ref = T.align6d_batch(d["particles"].numpy(), d["templates"].numpy(), S=w.n_shells,
                          r_max=w.r_max, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter, L_sched=w.L_sched,
                          rounds=w.rounds, max_shift=w.max_shift, upsample=10)
    parts, temps = d["particles"].cuda(), d["templates"].cuda()
    plan = m.plan_for_workload(w, precision=m.FP64)
    got = m.matcha_align6d(plan, parts, temps, w.rounds, w.max_shift, 10)
    torch.cuda.synchronize()
    for b in range(w.B):
        assert O.rotation_angle(got["R"][b].cpu().numpy(), ref["R"][b]) < 1e-8
        assert np.array_equal(got["t"][b].cpu().numpy(), ref["t"][b])
        assert np.abs(got["tau"][b].cpu().numpy() - ref["tau"][b]).max() < 1e-8
        assert abs(got["score"][b].item() - ref["score"][b]) <= 1e-10 * abs(ref["score"][b])
        assert abs(got["cc"][b].item() - ref["cc"][b]) <= 1e-10 * abs(ref["cc"][b])
        assert int(got["flags"][b]) == int(ref["flags"][b])
    plan.close()
    plan = m.plan_for_workload(w, precision=m.FP32)
    got = m.matcha_align6d(plan, parts, temps, w.rounds, w.max_shift, 10)
    torch.cuda.synchronize()
    for b in range(w.B):
        assert math.degrees(O.rotation_angle(got["R"][b].cpu().numpy(), ref["R"][b])) < 0.05
        assert np.abs(got["t"][b].cpu().numpy() - ref["t"][b]).max() <= 0.1 + 1e-12
    plan.close()


def test_align6d_full_batch_recovers_planted_poses():
    """The 1024-particle 64^3 batch with planted shifts up to 3 voxels, FP32:
    rotations and shifts against the planted pose, and two particles against
    the oracle's alternation."""
    w = W64
    d = synth.make_batch(w, device="cuda")
    plan = m.plan_for_workload(w, precision=m.FP32)
    got = m.matcha_align6d(plan, d["particles"], d["templates"], w.rounds, w.max_shift, 10)
    torch.cuda.synchronize()
    R = got["R"].cpu().numpy()
    tau = got["tau"].cpu().numpy()
    ang = np.degrees([O.rotation_angle(R[b], d["R_true"][b]) for b in range(w.B)])
    sh = np.abs(tau - d["tau_true"]).max(axis=1)
    print("6-D, 1024 x 64^3 FP32 vs planted: angle median %.3f p90 %.3f deg, shift median %.3f p90 %.3f vox"
          % (np.median(ang), np.percentile(ang, 90), np.median(sh), np.percentile(sh, 90)))
    assert np.median(ang) < 1.0 and np.median(sh) < 0.25
    sample = [0, 777]
    ref = T.align6d_batch(d["particles"][sample].cpu().numpy(), d["templates"][sample].cpu().numpy(),
                          S=w.n_shells, r_max=w.r_max, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter,
                          L_sched=w.L_sched, rounds=w.rounds, max_shift=w.max_shift, upsample=10)
    for i, b in enumerate(sample):
        assert math.degrees(O.rotation_angle(R[b], ref["R"][i])) < 0.05
        assert np.abs(got["t"][b].cpu().numpy() - ref["t"][i]).max() <= 0.1 + 1e-12
