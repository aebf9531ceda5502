"""The data-parallel path on two CPU ranks (gloo).

Particles are independent, so N GPUs shard the batch with no collective on the
data path; what needs checking is the host logic: disjoint contiguous shards
that reproduce the single-process batch, the timing barrier, and the
max-over-ranks time behind the whole-job rate.
"""
import socket

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
