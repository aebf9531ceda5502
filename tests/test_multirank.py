"""The data-parallel path on two CPU ranks (gloo).

Particles are independent, so N GPUs shard the batch with no collective on the
data path; what needs checking is the host logic: disjoint contiguous shards
that reproduce the single-process batch, the timing barrier, the
max-over-ranks time behind the whole-job rate, the cost-balanced (LPT) split
of an uneven batch, and the one all-reduce of a shared template's gradient.
"""
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import synth
from paper_2603_15285_gb300 import shard
import multirank_worker


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_start_and_rate_single_process():
    assert [shard.shard_start(r, 4) for r in range(3)] == [0, 4, 8]
    assert shard.max_over_ranks(2.5, 1) == 2.5
    assert shard.aggregate_rate(8, 1024, 2.0) == 4096.0


@pytest.mark.timeout(300)
def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    ws = 2
    mp.start_processes(multirank_worker.run, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       join=True, start_method="spawn")
    res = [torch.load(tmp_path / ("rank%d.pt" % r)) for r in range(ws)]
    for r in res:
        assert r["t_max"] == 2.0            # max of the ranks' 1.0 and 2.0
        assert r["rate"] == 2 * 2 / 2.0     # all ranks' particles over the slowest time
    # the ranks' shards, side by side, are the single-process batch
    w = synth.WORKLOADS["small32"]
    whole = synth.make_batch(w, B=4, start=0, device="cpu")["particles"]
    got = res[0]["gathered"].reshape(whole.shape)
    assert torch.equal(got, whole)
    assert torch.equal(res[0]["gathered"], res[1]["gathered"])


def test_lpt_shards_balance_and_cover():
    costs = [shard.particle_cost(P, L) for P, L in [(8, (8, 16, 24)), (32, (8, 16, 24, 32, 40, 48)),
                                                      (16, (8, 16, 24, 32)), (8, (8, 16, 24)),
                                                      (24, (8, 16, 24, 32, 40, 48)), (12, (8, 16))]]
    assert shard.wigner_terms(32) == 47905 and shard.particle_cost(16, (8, 16, 24, 32)) == 3659712
    for ws in (1, 2, 3):
        parts = shard.lpt_shards(costs, ws)
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT's bound: the largest load is at most 4/3 of the optimum, and the
        # optimum is at least the mean load and the largest single cost
        assert max(loads) <= 4.0 / 3.0 * max(sum(costs) / ws, max(costs)) + 1e-9
    assert shard.lpt_shards([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]


@pytest.mark.timeout(300)
def test_two_gloo_ranks_oracle_shards_and_gradient_allreduce(tmp_path):
    """Each rank aligns its LPT shard with the oracle and sums its particles'
    template gradients; after one all-reduce both ranks hold the gradient of
    the whole batch, equal bit for bit to a single process's (the same
    per-shard sums added in rank order)."""
    import oracle as O
    ws, n = 2, 5
    mp.start_processes(multirank_worker.run_oracle_shards, args=(ws, _free_port(), str(tmp_path), n),
                       nprocs=ws, join=True, start_method="spawn")
    res = [torch.load(tmp_path / ("oracle_rank%d.pt" % r), weights_only=False) for r in range(ws)]
    assert sorted(res[0]["idx"] + res[1]["idx"]) == list(range(n))
    small = dict(S=8, r_max=7.0, L0=4, K=1, M_iter=2, L_sched=(4, 6))
    d = synth.make_batch(synth.WORKLOADS["small32"], B=n, device="cpu")
    P_per = np.array([2 + (i * 5) % 4 for i in range(n)], dtype=np.int32)
    parts, temps = d["particles"].numpy(), d["templates"].numpy()[:1]
    ref = O.align_batch(parts, temps, P=4, P_per=P_per, n_threads=1, **small)
    L = small["L_sched"][-1]
    f = np.stack([O.analyze_volume(p, small["S"], small["r_max"], L) for p in parts])
    h = O.analyze_volume(temps[0], small["S"], small["r_max"], L)
    G, _, _ = O.template_grad_batch(f, h, ref["euler"], S=small["S"], r_max=small["r_max"],
                                    L_sched=list(small["L_sched"]), N=32, n_threads=1)
    for r in res:
        assert np.array_equal(r["euler"], ref["euler"][r["idx"]])
    total = G[res[0]["idx"]].sum(axis=0) + G[res[1]["idx"]].sum(axis=0)
    want = torch.view_as_real(torch.from_numpy(np.ascontiguousarray(total)))
    assert torch.equal(res[0]["grad"], want) and torch.equal(res[1]["grad"], want)
