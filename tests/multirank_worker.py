"""Worker of the two-rank CPU test (gloo): one process per rank."""
import datetime
import os


def run(rank, world_size, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    import synth
    from paper_2603_15285_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world_size,
                            timeout=datetime.timedelta(seconds=60))
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
