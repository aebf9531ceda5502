"""Workers of the two-rank CPU tests (gloo): one process per rank."""
import datetime
import os


def _init(rank, world_size, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world_size,
                            timeout=datetime.timedelta(seconds=120))


def run(rank, world_size, port, out_dir):
    import torch
    import torch.distributed as dist
    import synth
    from paper_2603_15285_gb300 import shard
    _init(rank, world_size, port)
    try:
        per_rank = 2
        w = synth.WORKLOADS["small32"]
        # each rank generates only its own particles
        d = synth.make_batch(w, B=per_rank, start=shard.shard_start(rank, per_rank), device="cpu")
        parts = d["particles"].contiguous()
        gathered = [torch.empty_like(parts) for _ in range(world_size)]
        dist.all_gather(gathered, parts)
        shard.barrier(world_size)
        # the slowest rank's time decides the job's rate
        t = 1.0 + rank
        t_max = shard.max_over_ranks(t, world_size)
        rate = shard.aggregate_rate(world_size, per_rank, t_max)
        torch.save({"gathered": torch.stack(gathered), "t_max": t_max, "rate": rate},
                   os.path.join(out_dir, "rank%d.pt" % rank))
    finally:
        dist.destroy_process_group()


def run_oracle_shards(rank, world_size, port, out_dir, n):
    """Each rank aligns its LPT shard of a mixed-cost batch with the oracle and
    adds its particles' template gradients; the gradient is summed over the
    ranks with one all-reduce."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle as O
    import synth
    from paper_2603_15285_gb300 import shard
    _init(rank, world_size, port)
    try:
        small = dict(S=8, r_max=7.0, L0=4, K=1, M_iter=2, L_sched=(4, 6))
        d = synth.make_batch(synth.WORKLOADS["small32"], B=n, device="cpu")
        P_per = np.array([2 + (i * 5) % 4 for i in range(n)], dtype=np.int32)
        costs = [shard.particle_cost(int(P_per[i]), small["L_sched"]) for i in range(n)]
        mine = shard.lpt_shards(costs, world_size)[rank]
        parts = d["particles"].numpy()[mine]
        temps = d["templates"].numpy()[:1]     # one shared template
        ref = O.align_batch(parts, temps, P=4, P_per=P_per[mine], n_threads=1, **small)
        L = small["L_sched"][-1]
        f = np.stack([O.analyze_volume(p, small["S"], small["r_max"], L) for p in parts])
        h = O.analyze_volume(temps[0], small["S"], small["r_max"], L)
        G, _, _ = O.template_grad_batch(f, h, ref["euler"], S=small["S"], r_max=small["r_max"],
                                        L_sched=list(small["L_sched"]), N=32, n_threads=1)
        g = torch.from_numpy(np.ascontiguousarray(G.sum(axis=0)))
        g = torch.view_as_real(g).contiguous()
        shard.allreduce_sum(g, world_size)
        torch.save({"idx": mine, "euler": ref["euler"], "grad": g},
                   os.path.join(out_dir, "oracle_rank%d.pt" % rank))
    finally:
        dist.destroy_process_group()
