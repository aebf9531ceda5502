"""Batches mixing box sizes (48^3, 64^3, 96^3 with their own shells and
bandwidths, per-particle SNR and candidate counts): the generator's
per-particle draws and the launch order of the groups (CPU)."""
import numpy as np

import synth
from paper_2603_15285_gb300 import mixed


def test_mixed_workloads_draw_per_particle_snr_and_P():
    for name, N in (("var48", 48), ("var64", 64), ("var96", 96)):
        w = synth.WORKLOADS[name]
        d = synth.make_batch(w, B=4, device="cpu", noise=False)
        assert tuple(d["particles"].shape) == (4, N, N, N)
        assert np.all((d["snr"] >= 0.05) & (d["snr"] <= 0.3))
        assert np.all((d["P_per"] >= 8) & (d["P_per"] <= 32))
        assert w.n_shells == w.L_sched[-1] and w.ball_radius == int(0.4 * N)


def test_groups_share_one_seed_sequence():
    # item 2048 of the mixed batch is particle 0 of the 64^3 group
    a = synth.WORKLOADS["var64"]
    assert a.seed_offset == 2048 and synth.WORKLOADS["var96"].seed_offset == 3072
    d0 = synth.make_batch(a, B=2, device="cpu", noise=False)
    d1 = synth.make_batch(a, B=1, start=1, device="cpu", noise=False)
    assert np.array_equal(d0["R_true"][1], d1["R_true"][0])


def test_groups_launch_most_expensive_first():
    costs = [mixed.group_cost(2048, 32, (8, 16, 24)), mixed.group_cost(1024, 32, (8, 16, 24, 32)),
             mixed.group_cost(1024, 32, (8, 16, 24, 32, 40, 48))]
    assert mixed.launch_order(costs) == [2, 1, 0]
    assert mixed.launch_order([1.0, 1.0, 2.0]) == [2, 0, 1]
