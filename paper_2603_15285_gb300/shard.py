"""Data-parallel sharding of independent particles across ranks.

Particles are independent units (every step of the alignment is per particle),
so a run on N GPUs gives each rank its own contiguous range of particles and
needs no collective on the data path: only the timing barrier and the
max-over-ranks of the elapsed time, which these helpers provide.  The same
helpers run on the ``nccl`` backend (CUDA tensors) and on ``gloo`` (CPU).
"""


def dist_env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    import os
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_start(rank: int, per_rank: int) -> int:
    """First particle index of `rank` when every rank aligns `per_rank` particles."""
    return rank * per_rank


def barrier(world_size: int):
    if world_size > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world_size: int, device="cpu") -> float:
    """The largest `value` over all ranks (the slowest rank's time)."""
    if world_size == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world_size: int, per_rank: int, seconds: float) -> float:
    """Whole-job throughput: all ranks' particles over the slowest rank's time."""
    return world_size * per_rank / seconds
